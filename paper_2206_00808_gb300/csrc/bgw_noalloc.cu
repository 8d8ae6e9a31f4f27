// Allocation-free matrix elements: bgw_mtxel_spinor_noalloc.
//
// Some callers cannot allocate device memory at the point where they need
// matrix elements: code running inside a memory pool or arena that owns all
// of the device's memory, plug-ins whose host application forbids
// cudaMalloc/cudaFree after start-up (both synchronise the device and can
// fail late), and real-time loops that must not block in the allocator.
// This entry point serves them: it runs the same kernels as the matrix-
// element stage of bgw_mtxel_spinor, but takes the real-space grids directly
// (no context) and keeps its scratch in one fixed, file-scope device array.
// It calls no cudaMalloc, cudaFree or any allocating library routine.
//
// The array holds BGW_NOALLOC_SCRATCH_BYTES and is part of the library image:
// every GPU that loads the library reserves it until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/bgw_chi.h"
#include "bgw_internal.h"

// Defined in bgw_api.cu: the message bgw_last_error(NULL) returns.
void bgw_set_global_error(const std::string &msg);

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[BGW_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
constexpr int kMaxNg = 65536;
constexpr int kMaxCube = 64 * 64 * 64;

struct DeviceSetup {
    bool done = false;
    void *scratch = nullptr;   // device address of g_noalloc_scratch
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Host staging of the sphere map (a static array, not heap or thread-local
// storage); g_map_mu serialises its use across host threads.
std::mutex g_map_mu;
int g_gmap_host[kMaxNg + kMaxCube];

bool supported_len(int n) {
    static const int lens[] = {16, 18, 20, 24, 27, 30, 32, 36, 40, 48, 64};
    for (int l : lens)
        if (l == n) return true;
    return false;
}

int pmod(long a, int n) {
    long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Once per device, with that device current: the FFT twiddle tables and the
// device address of the scratch array (the host-side name of the array is
// only a stand-in and must never reach a kernel).
bgw_status setup_device(int dev, void **scratch, std::string &err) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (dev < 0 || dev >= kMaxDevices) {
        err = "mtxel_noalloc: device index out of range";
        return BGW_E_ARG;
    }
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        cudaError_t e = bgw::grid_tables_init_f64();
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&s.scratch, g_noalloc_scratch);
        if (e != cudaSuccess) {
            err = std::string("mtxel_noalloc: device set-up: ") + cudaGetErrorString(e);
            s.scratch = nullptr;
            return BGW_E_CUDA;
        }
        s.done = true;
    }
    *scratch = s.scratch;
    return BGW_OK;
}

// A device pointer of the current device (or managed memory it can reach);
// cudaPointerGetAttributes allocates nothing.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" bgw_status bgw_mtxel_spinor_noalloc(const int fft[3], const void *Uv, const void *Uc,
                                               int nv, int nc, const int G0[3], int ng,
                                               const int *gvec, void *M_dev, void *stream) {
    std::string err;
    auto fail = [&](bgw_status s, const std::string &m) {
        bgw_set_global_error(m);
        return s;
    };
    if (!fft || !G0 || !gvec || !Uv || !Uc || !M_dev)
        return fail(BGW_E_ARG, "mtxel_noalloc: null pointer argument");
    for (int a = 0; a < 3; ++a)
        if (!supported_len(fft[a]))
            return fail(BGW_E_ARG, "mtxel_noalloc: FFT length " + std::to_string(fft[a]) + " not supported");
    if (nv < 0 || nc < 0) return fail(BGW_E_ARG, "mtxel_noalloc: negative band count");
    if (ng < 1 || ng > kMaxNg)
        return fail(BGW_E_ARG, "mtxel_noalloc: ng must be in 1.." + std::to_string(kMaxNg));
    // geometry of the dielectric sphere: kept widths and cube positions
    int emin[3], emax[3];
    for (int a = 0; a < 3; ++a) emin[a] = emax[a] = gvec[a];
    for (long g = 0; g < ng; ++g)
        for (int a = 0; a < 3; ++a) {
            emin[a] = std::min(emin[a], gvec[3 * g + a]);
            emax[a] = std::max(emax[a], gvec[3 * g + a]);
        }
    bgw::Axes ax;
    for (int a = 0; a < 3; ++a) {
        ax.n[a] = fft[a];
        ax.w[a] = std::min(emax[a] - emin[a] + 1, fft[a]);
        ax.s[a] = pmod((long)emin[a] + G0[a], fft[a]);
    }
    const long cube = (long)ax.w[0] * ax.w[1] * ax.w[2];
    const bool scatter = bgw::mtxel_scatter_mode(ax, 16);
    const long nmap = ng + (scatter ? cube : 0);
    const long P = (long)nv * nc;
    // Scratch of one block of vb valence bands: the sphere map, then the
    // kernels' z-pass (where used) and y-pass buffers for vb * nc pairs.  The
    // call runs in blocks of whole valence bands sized to the array.
    const size_t gbytes = round_up(sizeof(int) * (size_t)nmap);
    const size_t a_pair = bgw::mtxel_uses_a(ax) ? (size_t)fft[0] * fft[1] * ax.w[2] * 16 : 0;
    const size_t b_pair = (size_t)fft[0] * ax.w[1] * ax.w[2] * 16;
    auto need = [&](long vb) {
        const long pb = (long)std::min(vb, (long)bgw::mtxel_v_batch((int)vb, nc, ax, 16)) * nc;
        return gbytes + round_up((size_t)pb * a_pair) + round_up((size_t)pb * b_pair);
    };
    const size_t cap = (size_t)BGW_NOALLOC_SCRATCH_BYTES;
    if (P > 0 && need(1) > cap)
        return fail(BGW_E_ARG, "mtxel_noalloc: one valence band with " + std::to_string(nc) +
                                   " conduction bands needs " + std::to_string(need(1)) +
                                   " bytes of scratch, more than the " + std::to_string(cap) +
                                   "-byte maximum; split the conduction range");
    if (P == 0) return BGW_OK;
    long vb = nv;
    while (vb > 1 && need(vb) > cap) vb = std::max(1L, std::min(vb - 1, vb * (long)cap / (long)need(vb)));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(BGW_E_CUDA, std::string("mtxel_noalloc: ") + cudaGetErrorString(e));
    if (!on_device(Uv, dev) || !on_device(Uc, dev) || !on_device(M_dev, dev))
        return fail(BGW_E_ARG, "mtxel_noalloc: Uv, Uc and M_dev must be device memory of the current device " +
                                   std::to_string(dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The sphere map goes through a static host array: a captured copy would
    // read it at replay time, after later calls have rewritten it.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return fail(BGW_E_CUDA, std::string("mtxel_noalloc: ") + cudaGetErrorString(e));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(BGW_E_ARG, "mtxel_noalloc: the stream is being captured; this call cannot be captured");
    void *scratch = nullptr;
    const bgw_status s = setup_device(dev, &scratch, err);
    if (s != BGW_OK) return fail(s, err);
    std::lock_guard<std::mutex> lk(g_map_mu);
    for (long i = ng; i < nmap; ++i) g_gmap_host[i] = -1;
    for (long g = 0; g < ng; ++g) {
        int j[3];
        for (int a = 0; a < 3; ++a) j[a] = pmod((long)gvec[3 * g + a] - emin[a], fft[a]);
        const int cell = (j[0] * ax.w[1] + j[1]) * ax.w[2] + j[2];
        g_gmap_host[g] = cell;
        if (scatter) {
            if (g_gmap_host[ng + cell] >= 0)
                return fail(BGW_E_ARG, "mtxel_noalloc: aliased dielectric sphere too wide for the gather");
            g_gmap_host[ng + cell] = (int)g;
        }
    }
    char *base = static_cast<char *>(scratch);
    int *gmap = reinterpret_cast<int *>(base);
    const long pb = (long)std::min(vb, (long)bgw::mtxel_v_batch((int)vb, nc, ax, 16)) * nc;
    char *abuf = base + gbytes;
    char *bbuf = abuf + round_up((size_t)pb * a_pair);
    // pageable source: the copy waits for earlier work on the stream and has
    // read g_gmap_host when this call returns
    e = cudaMemcpyAsync(gmap, g_gmap_host, sizeof(int) * (size_t)nmap, cudaMemcpyHostToDevice, st);
    const long nbox = (long)fft[0] * fft[1] * fft[2];
    for (long v0 = 0; e == cudaSuccess && v0 < nv; v0 += vb) {
        const int n = (int)std::min(vb, (long)nv - v0);
        const void *uv = static_cast<const char *>(Uv) + (size_t)v0 * 2 * nbox * 16;
        void *m = static_cast<char *>(M_dev) + (size_t)v0 * nc * ng * 16;
        e = bgw::mtxel_f64(uv, Uc, n, nc, ax, gmap, ng, abuf, bbuf, m, ng, st);
    }
    if (e != cudaSuccess) return fail(BGW_E_CUDA, std::string("mtxel_noalloc: ") + cudaGetErrorString(e));
    return BGW_OK;
}
