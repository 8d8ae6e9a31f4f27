// C-ABI of libbgwchi.so (declared in include/bgw_chi.h): validation,
// geometry bookkeeping and the order of kernel launches for the spinor
// polarizability chi0_GG'(q, i omega) of arXiv:2206.00808, Sec. II.
//
// Data kept on the device by a context:
//   grids  [nk][nb][2][N1*N2*N3]  real-space spinor components u_nk,alpha(r)
//                                 (complex128 for FP64, complex64 for mixed)
//   energy [nk][nb]               band energies, eV
//   per q of the current q-set: gmap[ng] (position of each G in the kept
//   cube of the pruned forward FFT) and the FP64 accumulator
//   acc[nfreq][ng][ng] (lower block triangle filled; finalize mirrors it).
// Scratch buffers grow on demand and are reused.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <utility>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bgw_chi.h"
#include "bgw_internal.h"
#include "bgw_mixed.h"
#include "bgw_f64tc.h"

namespace {

thread_local std::string g_create_error;

// Allocation-failure injection for tests: when positive, the n-th device
// allocation from now on fails as if the device were out of memory (set by
// BGW_OPT_TEST_FAIL_ALLOC or the environment variable BGW_FAULT=oom@n).
std::atomic<long> g_fail_alloc{0};

cudaError_t dev_alloc(void **p, size_t bytes) {
    long n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    // Grow to at least `bytes`; old contents are not kept.  Waits for the
    // stream first so no queued kernel still reads the old allocation.
    cudaError_t ensure(size_t bytes, cudaStream_t st) {
        if (bytes <= cap) return cudaSuccess;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return cudaErrorNotPermitted;   // no allocation inside a graph capture
        if (p) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            cudaFree(p);
            p = nullptr;
            cap = 0;
        }
        cudaError_t e = dev_alloc(&p, bytes);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        cap = bytes;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

struct KPoint {
    bool uploaded = false;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};   // sphere extents (Miller)
    int ngw = 0;
    std::vector<int> cube_map;                  // host copy of the device map: cube cell ->
                                                // coefficient (or -1), then coefficient -> cell
    DevBuf map_dev;
    DevBuf coeff;                               // streaming mode: device copy of host coefficients
    const double *coeff_src = nullptr;          // streaming mode: coefficients the grid is built from
    int slot = -1;                              // grid slot holding this k (-1: none)
    const double *pending = nullptr;            // BGW_OPT_DEFER_K1: grid not built yet, from these
    // BGW_OPT_COPY_AHEAD: `coeff` is written on a copy stream; `copied`
    // marks that copy complete, `consumed` the last transform that read it;
    // copy_wait: a deferred build must make the context stream wait for it
    cudaEvent_t copied = nullptr, consumed = nullptr;
    bool consumed_set = false;
    bool copy_wait = false;
};

struct QState {
    double q[3];
    int ng = 0, nc = 0;
    std::vector<int> gvec;   // [ng][3]
    int emin[3], emax[3];
    int w[3];                // kept widths, min(emax - emin + 1, N)
    std::vector<int> gmap;   // [ng]
    std::vector<int> kmap;   // [nk]: grid index of k + q, -1 if off the grid
    DevBuf gmap_dev, kmap_dev;
    DevBuf acc;              // complex128 [nfreq][ng][ng]
};

bool is_supported_len(int n) {
    static const int lens[] = {16, 18, 20, 24, 27, 30, 32, 36, 40, 48, 64};
    for (int l : lens)
        if (l == n) return true;
    return false;
}

int pmod(long a, int n) {
    long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

// Device tables (FFT twiddles) are uploaded once per device per process.
std::mutex g_tables_mu;
bool g_tables_done[128];

cudaError_t ensure_tables(int dev) {
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (g_tables_done[dev]) return cudaSuccess;
    cudaError_t e = bgw::grid_tables_init_f64();
    if (e == cudaSuccess) e = bgw::grid_tables_init_f32();
    if (e == cudaSuccess) g_tables_done[dev] = true;
    return e;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

void bgw_set_global_error(const std::string &msg) { g_create_error = msg; }

struct bgw_ctx_s {
    int box[3];
    long nbox;
    int nk, nv, nc_max, nb;
    std::vector<double> kcrys;
    bgw_precision prec;
    cudaStream_t st;
    int device;
    size_t csize;        // bytes per complex grid / M element
    DevBuf grids, energy;
    std::vector<KPoint> k;
    DevBuf stage;        // host-uploaded coefficients
    DevBuf S, R;         // sphere -> grid scratch
    DevBuf A, Bs, M, W;  // mtxel scratch, M block, weights
    DevBuf mixed_ws;     // contraction workspace (split operands / FP64 partial sums)
    size_t M_half = 0;   // one half of M when the contraction is overlapped
    DevBuf freq_dev;
    DevBuf out_stage;    // finalize to host
    DevBuf gmap_tmp;     // dielectric-sphere map of a bgw_mtxel_spinor call
    DevBuf errflag;      // device int: non-zero after a bounded device wait gave up
    // scratch of the self-energy and BSE kernel calls (matrix-element blocks,
    // products, per-pair sums, a copy of the interaction's diagonal)
    DevBuf nx_m1, nx_m2, nx_y, nx_t, nx_s, nx_v;
    // real-space grid slots: every k resident (nslots == nk), or a
    // least-recently-used cache of nslots grids (streaming)
    int grid_slots_opt = 0;
    int nslots = 0;
    std::vector<int> slot_k;
    std::vector<long> slot_stamp;
    long use_clock = 0;
    bool streaming() const { return nslots > 0 && nslots < nk; }
    // graph capture (bgw_graph_*)
    bool capturing = false;
    cudaGraphExec_t gexec = nullptr;
    // tuning (bgw_set_option / bgw_autotune)
    int kchunk = 1;      // k-points per contraction launch
    int sm_count = 0;
    int tile_v = 0, tile_c = 0;   // pair tile of the FP32 plane kernel (0 = automatic)
    int test_drop_load = 0;       // BGW_OPT_TEST_DROP_LOAD
    int k1_path = 0;              // BGW_OPT_K1_PATH
    int mtxel_lanes = 0;          // BGW_OPT_MTXEL_LANES
    int mtxel_zy = 0;             // BGW_OPT_MTXEL_ZY
    int defer_k1 = 0;             // BGW_OPT_DEFER_K1
    int copy_ahead = 0;           // BGW_OPT_COPY_AHEAD
    static constexpr int kCopyStreams = 4;
    cudaStream_t cst[kCopyStreams] = {};   // copy streams of copy-ahead host uploads (k-point ik uses ik % 4)
    int overlap = 0;              // BGW_OPT_OVERLAP
    int f64_dfma = 0;             // BGW_OPT_FP64_CONTRACTION: 1 = FP64 FMA kernel, 0 = digit slices on tcgen05
    cudaStream_t gst = nullptr;   // contraction stream of the overlapped mixed path
    cudaEvent_t ov_fork = nullptr, ov_join = nullptr, ov_free[2] = {nullptr, nullptr};
    int npending = 0;             // uploads whose grid is not built yet
    // k-points summed into the running sum (accumulate calls made since the
    // q-set was installed; replays of a captured graph are not counted)
    std::vector<int> kcount;
    // stage timing (bgw_profile)
    static constexpr int kStages = 7;
    bool prof = false;
    struct Rec { int stage; long kernels; cudaEvent_t a, b; cudaStream_t s; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[kStages] = {0};
    long prof_calls[kStages] = {0}, prof_kernels[kStages] = {0};
    cudaEvent_t take_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    // Bracket a launch group; returns the index to close, or -1.
    int stage_begin(int stage) { return stage_begin_on(stage, st); }
    int stage_begin_on(int stage, cudaStream_t s) {
        if (!prof || capturing) return -1;
        Rec r{stage, 0, take_event(), take_event(), s};
        if (!r.a || !r.b) return -1;
        cudaEventRecord(r.a, s);
        recs.push_back(r);
        return (int)recs.size() - 1;
    }
    void stage_end(int idx, long kernels) {
        if (idx < 0) return;
        recs[idx].kernels = kernels;
        cudaEventRecord(recs[idx].b, recs[idx].s);
    }
    // Drop the last record opened if it is still the last one (nothing launched in it).
    void stage_cancel(int idx) {
        if (idx < 0 || idx != (int)recs.size() - 1) return;
        pool.push_back(recs.back().a);
        pool.push_back(recs.back().b);
        recs.pop_back();
    }
    // Fold finished records into the totals (blocks on the stream).
    cudaError_t drain() {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        for (auto &r : recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) prof_ms[r.stage] += ms;
            prof_calls[r.stage] += 1;
            prof_kernels[r.stage] += r.kernels;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
        return cudaSuccess;
    }
    // current q-set of the accumulators
    bool have_qset = false;
    int nfreq = 0;
    std::vector<double> freq;
    std::vector<QState> qs;
    std::string err;

    bgw_status fail(bgw_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
    bgw_status cuda_fail(cudaError_t e, const char *what) {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        if (e == cudaErrorNotPermitted && capturing)
            err += " (a buffer would have to grow during graph capture: run the same calls once "
                   "before bgw_graph_begin)";
        return e == cudaErrorMemoryAllocation ? BGW_E_NOMEM : BGW_E_CUDA;
    }
    long grid_elems_per_k() const { return (long)nb * 2 * nbox; }
    char *slot_ptr(int slot, int band) {
        return static_cast<char *>(grids.p) + ((long)slot * grid_elems_per_k() + (long)band * 2 * nbox) * csize;
    }
};

#include <cstdarg>
bgw_status bgw_ctx_s::fail(bgw_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return s;
}

namespace {

// Grid slots are allocated at the first upload: every k (default) or the
// BGW_OPT_GRID_SLOTS most recently used ones.
cudaError_t ensure_slots(bgw_ctx_s *c) {
    if (c->nslots > 0) return cudaSuccess;
    const int n = (c->grid_slots_opt > 0 && c->grid_slots_opt < c->nk) ? std::max(2, c->grid_slots_opt)
                                                                         : c->nk;
    cudaError_t e = c->grids.ensure((size_t)n * c->grid_elems_per_k() * c->csize, c->st);
    if (e != cudaSuccess) return e;
    c->nslots = n;
    c->slot_k.assign(n, -1);
    c->slot_stamp.assign(n, 0);
    return cudaSuccess;
}

// Sphere -> real-space grid of every band of k into grid slot `slot`.
cudaError_t run_k1(bgw_ctx_s *c, int ik, const double *src, int slot) {
    KPoint &kp = c->k[ik];
    const long B = 2L * c->nb;
    int w[3];
    for (int a = 0; a < 3; ++a) w[a] = kp.hi[a] - kp.lo[a] + 1;
    const size_t sbytes = (size_t)B * c->box[0] * w[1] * w[2] * c->csize;
    bgw::Axes ax;
    for (int a = 0; a < 3; ++a) {
        ax.n[a] = c->box[a];
        ax.w[a] = w[a];
        ax.s[a] = pmod(kp.lo[a], c->box[a]);
    }
    const size_t rbytes =
        bgw::wfn_uses_r(ax, c->csize) ? (size_t)B * c->box[0] * c->box[1] * w[2] * c->csize : 0;
    cudaError_t e = c->S.ensure(sbytes, c->st);
    if (e == cudaSuccess) e = c->R.ensure(rbytes, c->st);
    if (e != cudaSuccess) return e;
    void *U = c->slot_ptr(slot, 0);
    const int *mp = static_cast<const int *>(kp.map_dev.p);
    const int rec = c->stage_begin(0);
    e = (c->prec == BGW_FP64)
            ? bgw::wfn_to_grid_f64(src, kp.ngw, (int)B, mp, ax, c->S.p, c->R.p, U, c->st, c->k1_path)
            : bgw::wfn_to_grid_f32(src, kp.ngw, (int)B, mp, ax, c->S.p, c->R.p, U, c->st, c->k1_path);
    c->stage_end(rec, 3);
    return e;
}

// Grid slot of k: resident mode, slot k; streaming, the k's slot if cached,
// else the least recently used slot is rebuilt from the stored coefficients.
// Every use and rebuild is queued on the one context stream, so a slot is
// never overwritten before the kernels that read it have run.
int ensure_grid(bgw_ctx_s *c, int ik, cudaError_t &e) {
    e = cudaSuccess;
    if (!c->streaming()) return ik;
    KPoint &kp = c->k[ik];
    if (kp.slot < 0) {
        int victim = 0;
        for (int i = 1; i < c->nslots; ++i)
            if (c->slot_stamp[i] < c->slot_stamp[victim]) victim = i;
        if (c->slot_k[victim] >= 0) c->k[c->slot_k[victim]].slot = -1;
        c->slot_k[victim] = ik;
        kp.slot = victim;
        e = run_k1(c, ik, kp.coeff_src, victim);
        if (e != cudaSuccess) {
            c->slot_k[victim] = -1;
            kp.slot = -1;
            return -1;
        }
    }
    c->slot_stamp[kp.slot] = ++c->use_clock;
    return kp.slot;
}

// The context stream is being captured (through bgw_graph_begin or by the
// caller): copy-ahead then falls back to copies on the context stream.
bool st_capturing(const bgw_ctx_s *c) {
    if (c->capturing) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return c->st && cudaStreamIsCapturing(c->st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Copy-ahead host uploads: the copy stream and the k-point's two events.
cudaError_t ensure_copy_events(bgw_ctx_s *c, KPoint &kp) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < bgw_ctx_s::kCopyStreams && e == cudaSuccess; ++i)
        if (!c->cst[i]) e = cudaStreamCreateWithFlags(&c->cst[i], cudaStreamNonBlocking);
    if (e == cudaSuccess && !kp.copied) e = cudaEventCreateWithFlags(&kp.copied, cudaEventDisableTiming);
    if (e == cudaSuccess && !kp.consumed) e = cudaEventCreateWithFlags(&kp.consumed, cudaEventDisableTiming);
    return e;
}

// Marks the end of the kernels that read k's device coefficients, for the
// next copy-ahead copy into the same buffer.  Inside a graph capture the
// graph's launches are marked instead (bgw_graph_launch).
cudaError_t mark_consumed(bgw_ctx_s *c, KPoint &kp) {
    if (!kp.consumed || st_capturing(c)) return cudaSuccess;
    kp.consumed_set = true;
    return cudaEventRecord(kp.consumed, c->st);
}

// Builds the grids of the deferred uploads (BGW_OPT_DEFER_K1): one launch
// per up to 64 k-points where every pending k takes the one-kernel transform
// of the automatic path, else one run_k1 per k.  Queued on the context
// stream ahead of the kernels that read the grids.
cudaError_t flush_k1(bgw_ctx_s *c) {
    if (c->npending == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    std::vector<bgw::K1Job> jobs;
    std::vector<int> ks;
    for (int ik = 0; ik < c->nk; ++ik) {
        KPoint &kp = c->k[ik];
        if (!kp.pending) continue;
        bgw::K1Job j;
        j.coeff = kp.pending;
        j.ngw = kp.ngw;
        j.cube_map = static_cast<const int *>(kp.map_dev.p);
        for (int a = 0; a < 3; ++a) {
            j.a.n[a] = c->box[a];
            j.a.w[a] = kp.hi[a] - kp.lo[a] + 1;
            j.a.s[a] = pmod(kp.lo[a], c->box[a]);
        }
        j.U = c->slot_ptr(ik, 0);
        jobs.push_back(j);
        ks.push_back(ik);
    }
    // copy-ahead uploads of these k-points: the builds wait for their copies
    for (int ik : ks) {
        KPoint &kp = c->k[ik];
        if (kp.copy_wait && e == cudaSuccess) e = cudaStreamWaitEvent(c->st, kp.copied, 0);
        kp.copy_wait = false;
    }
    if (e != cudaSuccess) return e;
    bool batched = false;
    if (c->k1_path == 0) {
        const int rec = c->stage_begin(0);
        const int B = 2 * c->nb;
        e = (c->prec == BGW_FP64) ? bgw::wfn_to_grid_batch_f64(jobs.data(), (int)jobs.size(), B, c->st, &batched)
                                  : bgw::wfn_to_grid_batch_f32(jobs.data(), (int)jobs.size(), B, c->st, &batched);
        c->stage_end(rec, batched ? (long)((jobs.size() + 63) / 64) : 0);
    }
    for (size_t i = 0; e == cudaSuccess && !batched && i < ks.size(); ++i)
        e = run_k1(c, ks[i], jobs[i].coeff, ks[i]);
    for (size_t i = 0; e == cudaSuccess && i < ks.size(); ++i) e = mark_consumed(c, c->k[ks[i]]);
    if (e != cudaSuccess) return e;
    for (int ik : ks) c->k[ik].pending = nullptr;
    c->npending = 0;
    return cudaSuccess;
}

// k + q = k' + G0 with k' on the list (tolerance 1e-6 in crystal units).
bool find_umklapp(const bgw_ctx_s *c, int ik, const double q[3], int &kp, int G0[3]) {
    for (int j = 0; j < c->nk; ++j) {
        bool ok = true;
        int g[3];
        for (int a = 0; a < 3; ++a) {
            const double d = c->kcrys[3 * ik + a] + q[a] - c->kcrys[3 * j + a];
            const double r = std::nearbyint(d);
            if (std::fabs(d - r) > 1e-6) {
                ok = false;
                break;
            }
            g[a] = (int)r;
        }
        if (ok) {
            kp = j;
            for (int a = 0; a < 3; ++a) G0[a] = g[a];
            return true;
        }
    }
    return false;
}

void compute_kmap(const bgw_ctx_s *c, QState &s);

// Geometry of one dielectric sphere: extents, kept widths, cube positions.
bgw_status prepare_q(bgw_ctx_s *c, const bgw_q *q, QState &s, bool check_nc = true) {
    if (!q) return c->fail(BGW_E_ARG, "null q");
    if (q->ng < 1 || !q->gvec) return c->fail(BGW_E_ARG, "q: ng must be >= 1 with a gvec list");
    if (check_nc && (q->nc < 1 || q->nc > c->nc_max))
        return c->fail(BGW_E_ARG, "q: nc=%d outside 1..nc_max=%d", q->nc, c->nc_max);
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(q->q[a])) return c->fail(BGW_E_ARG, "q: non-finite component");
        s.q[a] = q->q[a];
    }
    s.ng = q->ng;
    s.nc = q->nc;
    s.gvec.assign(q->gvec, q->gvec + 3 * (long)q->ng);
    for (int a = 0; a < 3; ++a) {
        s.emin[a] = s.emax[a] = s.gvec[a];
    }
    for (int g = 0; g < s.ng; ++g)
        for (int a = 0; a < 3; ++a) {
            s.emin[a] = std::min(s.emin[a], s.gvec[3 * g + a]);
            s.emax[a] = std::max(s.emax[a], s.gvec[3 * g + a]);
        }
    for (int a = 0; a < 3; ++a) s.w[a] = std::min(s.emax[a] - s.emin[a] + 1, c->box[a]);
    const long cube = (long)s.w[0] * s.w[1] * s.w[2];
    bgw::Axes ax;
    for (int a = 0; a < 3; ++a) {
        ax.n[a] = c->box[a];
        ax.w[a] = s.w[a];
        ax.s[a] = 0;
    }
    const bool scatter = bgw::mtxel_scatter_mode(ax, c->csize);
    // Two G that agree mod N (an aliased sphere) share a cube cell and both
    // read the same cyclic value, which is what the FFT route gives.
    s.gmap.assign(s.ng + (scatter ? cube : 0), -1);
    for (int g = 0; g < s.ng; ++g) {
        int j[3];
        for (int a = 0; a < 3; ++a) j[a] = pmod((long)s.gvec[3 * g + a] - s.emin[a], c->box[a]);
        const int cell = (j[0] * s.w[1] + j[1]) * s.w[2] + j[2];
        s.gmap[g] = cell;
        if (scatter) {
            if (s.gmap[s.ng + cell] >= 0)
                return c->fail(BGW_E_ARG, "dielectric sphere aliased on this box (two G share a cell) "
                                          "and too wide (%dx%dx%d) for the shared-memory gather",
                               s.w[0], s.w[1], s.w[2]);
            s.gmap[s.ng + cell] = g;
        }
    }
    compute_kmap(c, s);
    return BGW_OK;
}

bool same_q(const QState &s, const bgw_q *q) {
    if (s.ng != q->ng || s.nc != q->nc) return false;
    for (int a = 0; a < 3; ++a)
        if (s.q[a] != q->q[a]) return false;
    return std::equal(s.gvec.begin(), s.gvec.end(), q->gvec);
}

// Alias-free test for one (k, k+q) pair of spheres and one dielectric sphere:
// the product density has Fourier components h2 - h1 in [dmin, dmax]; no
// other component folds onto a G in [emin, emax] iff N > dmax - emin and
// N > emax - dmin on every axis.
bool alias_free(const bgw_ctx_s *c, int ik, int kp, const int G0[3], const QState &s) {
    for (int a = 0; a < 3; ++a) {
        const int dmin = (c->k[kp].lo[a] - G0[a]) - c->k[ik].hi[a];
        const int dmax = (c->k[kp].hi[a] - G0[a]) - c->k[ik].lo[a];
        if (!(c->box[a] > dmax - s.emin[a] && c->box[a] > s.emax[a] - dmin)) return false;
    }
    return true;
}

bgw::Axes mtxel_axes(const bgw_ctx_s *c, const QState &s, const int G0[3]) {
    bgw::Axes ax;
    for (int a = 0; a < 3; ++a) {
        ax.n[a] = c->box[a];
        ax.w[a] = s.w[a];
        ax.s[a] = pmod((long)s.emin[a] + G0[a], c->box[a]);
    }
    return ax;
}

// Scratch of the matrix-element kernels for one k of q-point s (P = nv x nc
// pairs, processed in batches of whole valence bands).
cudaError_t ensure_mtxel_scratch(bgw_ctx_s *c, const QState &s, long P) {
    const long n01 = (long)c->box[0] * c->box[1];
    const int G0z[3] = {0, 0, 0};
    const bgw::Axes ax = mtxel_axes(c, s, G0z);
    if (P > 0) {
        const int nc = (int)(P / c->nv);
        P = (long)bgw::mtxel_v_batch((int)(P / std::max(1, nc)), nc, ax, c->csize) * nc;
    }
    const long PA = bgw::mtxel_uses_a(ax) ? P : 0;
    cudaError_t e = c->A.ensure((size_t)(PA * n01 * s.w[2]) * c->csize, c->st);
    if (e == cudaSuccess) e = c->Bs.ensure((size_t)(P * c->box[0] * s.w[1] * s.w[2]) * c->csize, c->st);
    return e;
}

// Profiling of the matrix-element kernels in two stages: 1 the pair density
// with the z and y passes, 6 the x pass with the sphere gather.  The hook
// closes the open record and opens one of the other stage at each x-pass mark.
struct XProf {
    bgw_ctx_s *c;
    int rec;
    bgw::XPassHook hook;
    explicit XProf(bgw_ctx_s *ctx) : c(ctx), rec(ctx->stage_begin(1)), hook{&XProf::mark, this} {}
    const bgw::XPassHook *get() const { return rec >= 0 ? &hook : nullptr; }
    void finish() { c->stage_cancel(rec); }
    static void mark(void *p, int begin, int kernels) {
        auto *x = static_cast<XProf *>(p);
        x->c->stage_end(x->rec, kernels);
        x->rec = x->c->stage_begin(begin ? 6 : 1);
    }
};

cudaError_t launch_mtxel(bgw_ctx_s *c, const QState &s, int ik, int kp, const int G0[3], int v0,
                         int nv, int c0, int nc, void *M, long ldm, int tv = 0, int tc = 0) {
    const bgw::Axes ax = mtxel_axes(c, s, G0);
    cudaError_t ge;
    const int sv = ensure_grid(c, ik, ge);
    if (ge != cudaSuccess) return ge;
    const int sc = ensure_grid(c, kp, ge);
    if (ge != cudaSuccess) return ge;
    const void *Uv = c->slot_ptr(sv, v0);
    const void *Uc = c->slot_ptr(sc, c->nv + c0);
    const int *gmap = static_cast<const int *>(s.gmap_dev.p);
    XProf xp(c);
    cudaError_t e = (c->prec == BGW_FP64)
        ? bgw::mtxel_f64(Uv, Uc, nv, nc, ax, gmap, s.ng, c->A.p, c->Bs.p, M, ldm, c->st, 0, 0, c->mtxel_lanes, 0,
                         xp.get())
        : bgw::mtxel_f32(Uv, Uc, nv, nc, ax, gmap, s.ng, c->A.p, c->Bs.p, M, ldm, c->st, tv, tc, c->mtxel_lanes,
                         c->mtxel_zy, xp.get(), static_cast<int *>(c->errflag.p), c->test_drop_load == 2);
    xp.finish();
    return e;
}


// Checks shared by accumulate and autotune; fills `fresh` with the q geometry.
bgw_status validate_qset(bgw_ctx_s *c, const char *who, int nq, const bgw_q *qs, int nfreq,
                         const double *freq_eV, int k_begin, int k_end, std::vector<QState> &fresh) {
    if (nq < 1 || !qs) return c->fail(BGW_E_ARG, "%s: nq >= 1 and a q list required", who);
    if (nfreq < 1 || !freq_eV) return c->fail(BGW_E_ARG, "%s: nfreq >= 1 and freq required", who);
    for (int j = 0; j < nfreq; ++j)
        if (!std::isfinite(freq_eV[j]) || freq_eV[j] < 0)
            return c->fail(BGW_E_ARG, "%s: frequency %d must be finite and >= 0", who, j);
    if (k_begin < 0 || k_end > c->nk || k_begin > k_end)
        return c->fail(BGW_E_ARG, "%s: k range [%d,%d) outside [0,%d)", who, k_begin, k_end, c->nk);
    fresh.assign(nq, QState());
    for (int iq = 0; iq < nq; ++iq) {
        bgw_status st = prepare_q(c, &qs[iq], fresh[iq]);
        if (st != BGW_OK) return st;
        for (int ik = k_begin; ik < k_end; ++ik) {
            const int kp = fresh[iq].kmap[ik];
            if (kp < 0) return c->fail(BGW_E_ARG, "%s: k + q not on the k list (q %d, k %d)", who, iq, ik);
            if (!c->k[ik].uploaded || !c->k[kp].uploaded)
                return c->fail(BGW_E_STATE, "%s: k %d or its partner %d not uploaded", who, ik, kp);
        }
    }
    return BGW_OK;
}

// kmap[k]: grid index of k + q for every k (-1 where k + q is off the grid).
void compute_kmap(const bgw_ctx_s *c, QState &s) {
    s.kmap.assign(c->nk, -1);
    for (int k = 0; k < c->nk; ++k) {
        int kp, G0[3];
        if (find_umklapp(c, k, s.q, kp, G0)) s.kmap[k] = kp;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }


// Bytes of split operands the mixed contraction keeps for q-point s.
size_t mixed_q_bytes(const bgw_ctx_s *c, const QState &s, int nfreq, int kchunk) {
    return align256(bgw::mixed_workspace_bytes((long)kchunk * c->nv * s.nc, s.ng, nfreq, (int)c->prec));
}

// Workspace of the FP64 contraction of P pairs (either kernel).
size_t f64_ws_bytes(const bgw_ctx_s *c, long P, int ng, int nfreq) {
    return c->f64_dfma ? bgw::herk_f64_workspace_bytes((int)P, ng, nfreq, c->sm_count)
                       : bgw::f64tc_workspace_bytes(P, ng, nfreq);
}

// Consecutive q-points contracted by one grouped launch (mixed path): at
// most mixed_max_group() of them and, past the first, no more than
// kGroupBytes of split operands.  FP64: one q per group.
constexpr size_t kGroupBytes = (size_t)4 << 30;

std::vector<std::pair<size_t, size_t>> form_groups(const bgw_ctx_s *c, const std::vector<QState> &qs,
                                                   int nfreq, int kchunk) {
    std::vector<std::pair<size_t, size_t>> groups;
    const size_t G = c->prec == BGW_FP64 ? 1 : (size_t)bgw::mixed_max_group();
    size_t b = 0;
    while (b < qs.size()) {
        size_t e = b, bytes = 0;
        while (e < qs.size() && e - b < G) {
            const size_t qb = c->prec == BGW_FP64 ? 0 : mixed_q_bytes(c, qs[e], nfreq, kchunk);
            if (e > b && bytes + qb > kGroupBytes) break;
            bytes += qb;
            ++e;
        }
        groups.emplace_back(b, e);
        b = e;
    }
    return groups;
}

// The mixed contraction overlaps the next block's matrix elements
// (BGW_OPT_OVERLAP): M in two halves, weights, split and contraction on
// their own stream.
bool overlapped(const bgw_ctx_s *c) { return c->overlap && c->prec != BGW_FP64; }

cudaError_t ensure_overlap_stream(bgw_ctx_s *c) {
    cudaError_t e = cudaSuccess;
    if (!c->gst) {
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->gst, cudaStreamNonBlocking, hi);
    }
    cudaEvent_t *evs[] = {&c->ov_fork, &c->ov_join, &c->ov_free[0], &c->ov_free[1]};
    for (cudaEvent_t *ev : evs)
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    return e;
}

// Scratch for contraction launches of up to kchunk k-points on every q
// (mixed: the split operands of a whole group of q-points at once).
cudaError_t ensure_chunk_scratch(bgw_ctx_s *c, const std::vector<QState> &qs, int nfreq, int kchunk) {
    long Pmax = 0, Mbytes = 0;
    size_t ws = 0;
    cudaError_t e = cudaSuccess;
    for (auto &gr : form_groups(c, qs, nfreq, kchunk)) {
        size_t sum = 0;
        for (size_t i = gr.first; i < gr.second; ++i) {
            const QState &s = qs[i];
            if (c->prec != BGW_FP64)
                sum += mixed_q_bytes(c, s, nfreq, kchunk);
            else
                sum = std::max(sum, f64_ws_bytes(c, (long)kchunk * c->nv * s.nc, s.ng, nfreq));
        }
        ws = std::max(ws, sum);
    }
    for (auto &s : qs) {
        const long P = (long)c->nv * s.nc;
        Pmax = std::max(Pmax, P);
        Mbytes = std::max(Mbytes, (long)kchunk * P * s.ng * (long)c->csize);
        e = ensure_mtxel_scratch(c, s, P);
        if (e != cudaSuccess) return e;
    }
    const size_t mhalf = align256((size_t)Mbytes);
    e = c->M.ensure(overlapped(c) ? 2 * mhalf : mhalf, c->st);
    if (e == cudaSuccess) c->M_half = mhalf;
    if (e == cudaSuccess) e = c->W.ensure(sizeof(double) * (size_t)kchunk * Pmax * nfreq, c->st);
    if (e == cudaSuccess && ws) e = c->mixed_ws.ensure(ws, c->st);
    return e;
}

// Make `fresh` the context's q-set: accumulators zeroed on the stream, the
// sphere and k maps on the device.  Buffers of the previous set are reused
// when the sizes agree, and nothing is copied from the host when the
// contents agree too (so repeated steps queue only a memset).
bgw_status install_qset(bgw_ctx_s *c, std::vector<QState> &fresh, int nfreq, const double *freq) {
    cudaError_t e = cudaSuccess;
    bool reuse = c->qs.size() == fresh.size() && c->nfreq == nfreq;
    for (size_t i = 0; reuse && i < fresh.size(); ++i)
        reuse = c->qs[i].ng == fresh[i].ng && c->qs[i].acc.p != nullptr;
    bool same_content = reuse && std::equal(c->freq.begin(), c->freq.end(), freq);
    for (size_t i = 0; same_content && i < fresh.size(); ++i)
        same_content = c->qs[i].gmap == fresh[i].gmap && c->qs[i].kmap == fresh[i].kmap;
    if (reuse) {
        for (size_t i = 0; i < fresh.size(); ++i) {
            std::swap(fresh[i].gmap_dev, c->qs[i].gmap_dev);
            std::swap(fresh[i].kmap_dev, c->qs[i].kmap_dev);
            std::swap(fresh[i].acc, c->qs[i].acc);
        }
    } else if (!c->qs.empty()) {
        e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "accumulate: stream");
        for (auto &s : c->qs) {
            s.gmap_dev.release();
            s.kmap_dev.release();
            s.acc.release();
        }
    }
    for (auto &s : fresh) {
        e = s.gmap_dev.ensure(sizeof(int) * s.gmap.size(), c->st);
        if (e == cudaSuccess) e = s.kmap_dev.ensure(sizeof(int) * (size_t)c->nk, c->st);
        if (e == cudaSuccess) e = s.acc.ensure(16 * (size_t)nfreq * s.ng * s.ng, c->st);
        if (e != cudaSuccess) {
            for (auto &t : fresh) {
                t.gmap_dev.release();
                t.kmap_dev.release();
                t.acc.release();
            }
            c->qs.clear();
            return c->cuda_fail(e, "accumulate: accumulators");
        }
    }
    e = c->freq_dev.ensure(sizeof(double) * nfreq, c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "accumulate: frequency buffer");
    c->qs.swap(fresh);
    c->freq.assign(freq, freq + nfreq);
    c->nfreq = nfreq;
    c->have_qset = true;
    c->kcount.assign(c->nk, 0);
    if (!same_content) {
        e = cudaMemcpyAsync(c->freq_dev.p, c->freq.data(), sizeof(double) * nfreq,
                            cudaMemcpyHostToDevice, c->st);
        for (auto &s : c->qs) {
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s.gmap_dev.p, s.gmap.data(), sizeof(int) * s.gmap.size(),
                                    cudaMemcpyHostToDevice, c->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s.kmap_dev.p, s.kmap.data(), sizeof(int) * c->nk,
                                    cudaMemcpyHostToDevice, c->st);
        }
    }
    for (auto &s : c->qs)
        if (e == cudaSuccess) e = cudaMemsetAsync(s.acc.p, 0, 16 * (size_t)nfreq * s.ng * s.ng, c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "accumulate: initialising accumulators");
    return BGW_OK;
}

// The k loop of bgw_chi0_accumulate for the given q-states.  Per chunk of
// kchunk k-points and per q: matrix elements of each k into consecutive M
// blocks and one weights launch; then FP64: one contraction launch per q;
// mixed: one operand split per q into its own workspace slice and ONE
// persistent grouped contraction for a whole group of q-points.
cudaError_t run_range(bgw_ctx_s *c, std::vector<QState> &qs, int nfreq, const double *freq,
                      int k_begin, int k_end, int kchunk, int tv, int tc, bool &clean) {
    cudaError_t e = cudaSuccess;
    const double *energy = static_cast<const double *>(c->energy.p);
    const auto groups = form_groups(c, qs, nfreq, kchunk);
    std::vector<bgw::MixedQ> group;
    // Overlapped (mixed): the matrix elements stay on the context stream and
    // write M blocks alternately into two halves of M; weights, split and
    // contraction run in order on the contraction stream, each block forked
    // after its matrix elements, and the matrix elements of a block wait for
    // the split that last read their half.  Every accumulator sees the same
    // launches in the same order as on one stream.
    const bool ovl = overlapped(c);
    if (ovl) {
        e = ensure_overlap_stream(c);
        if (e != cudaSuccess) return e;
    }
    cudaStream_t gs = ovl ? c->gst : c->st;
    bool half_used[2] = {false, false};
    int turn = 0;
    bool joined = true;
    auto join = [&]() -> cudaError_t {
        if (joined) return cudaSuccess;
        joined = true;
        cudaError_t r = cudaEventRecord(c->ov_join, c->gst);
        return r == cudaSuccess ? cudaStreamWaitEvent(c->st, c->ov_join, 0) : r;
    };
    for (int k0 = k_begin; k0 < k_end; k0 += kchunk) {
        const int kn = std::min(kchunk, k_end - k0);
        for (auto &gr : groups) {
            group.clear();
            size_t off = 0;
            for (size_t iq = gr.first; iq < gr.second; ++iq) {
                QState &s = qs[iq];
                const long P = (long)c->nv * s.nc;
                char *M = static_cast<char *>(c->M.p) + (ovl ? (size_t)turn * c->M_half : 0);
                if (ovl && half_used[turn]) {
                    e = cudaStreamWaitEvent(c->st, c->ov_free[turn], 0);
                    if (e != cudaSuccess) return join(), e;
                }
                for (int kl = 0; kl < kn; ++kl) {
                    const int ik = k0 + kl;
                    int kp, G0[3];
                    find_umklapp(c, ik, s.q, kp, G0);
                    clean = clean && alias_free(c, ik, kp, G0, s);
                    char *Mk = M + (size_t)kl * P * s.ng * c->csize;
                    e = launch_mtxel(c, s, ik, kp, G0, 0, c->nv, 0, s.nc, Mk, s.ng, tv, tc);
                    if (e != cudaSuccess) return join(), e;
                }
                if (ovl) {
                    e = cudaEventRecord(c->ov_fork, c->st);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, c->ov_fork, 0);
                    if (e != cudaSuccess) return join(), e;
                    joined = false;
                }
                const int PT = (int)(P * kn);
                {
                    const int rec = c->stage_begin_on(2, gs);
                    e = bgw::pair_weights(energy, c->nb, c->nv, s.nc, static_cast<const int *>(s.kmap_dev.p),
                                          k0, kn, freq, nfreq, static_cast<double *>(c->W.p), gs);
                    c->stage_end(rec, 1);
                    if (e != cudaSuccess) return join(), e;
                }
                if (c->prec == BGW_FP64) {
                    const int rec = c->stage_begin(3);
                    if (c->f64_dfma)
                        e = bgw::herk_f64(M, PT, s.ng, static_cast<const double *>(c->W.p), nfreq,
                                          s.acc.p, c->mixed_ws.p, c->sm_count, c->st);
                    else
                        e = bgw::f64tc_contract(M, PT, s.ng, static_cast<const double *>(c->W.p), nfreq, s.acc.p,
                                                c->mixed_ws.p, c->sm_count, c->st, static_cast<int *>(c->errflag.p));
                    c->stage_end(rec, c->f64_dfma ? 2 : 3);
                    if (e != cudaSuccess) return join(), e;
                } else {
                    void *ws = static_cast<char *>(c->mixed_ws.p) + off;
                    off += mixed_q_bytes(c, s, nfreq, kchunk);
                    const int rec = c->stage_begin_on(5, gs);
                    e = bgw::mixed_split(M, PT, s.ng, static_cast<const double *>(c->W.p), nfreq, ws, (int)c->prec,
                                         gs);
                    c->stage_end(rec, 1);
                    if (e == cudaSuccess && ovl) e = cudaEventRecord(c->ov_free[turn], gs);
                    if (e != cudaSuccess) return join(), e;
                    if (ovl) {
                        half_used[turn] = true;
                        turn ^= 1;
                    }
                    group.push_back(bgw::MixedQ{ws, PT, s.ng, s.acc.p});
                }
            }
            if (c->prec != BGW_FP64) {
                const int rec = c->stage_begin_on(3, gs);
                e = bgw::mixed_gemm(group.data(), (int)group.size(), nfreq, (int)c->prec, c->sm_count, gs,
                                    static_cast<int *>(c->errflag.p), c->test_drop_load == 1);
                c->stage_end(rec, 1);
                if (e != cudaSuccess) return join(), e;
            }
        }
    }
    cudaError_t ej = join();
    return e != cudaSuccess ? e : ej;
}
}  // namespace

// ---- matrix elements of any band ranges (self-energy, BSE kernel) ----------
namespace {

// Scratch of the matrix-element kernels for na x nb2 pairs of sphere s.
cudaError_t ensure_mtxel_scratch_pairs(bgw_ctx_s *c, const QState &s, int na, int nb2) {
    const long n01 = (long)c->box[0] * c->box[1];
    const int G0z[3] = {0, 0, 0};
    const bgw::Axes ax = mtxel_axes(c, s, G0z);
    const long P = (long)bgw::mtxel_v_batch(na, nb2, ax, c->csize) * nb2;
    const long PA = bgw::mtxel_uses_a(ax) ? P : 0;
    cudaError_t e = c->A.ensure((size_t)(PA * n01 * s.w[2]) * c->csize, c->st);
    if (e == cudaSuccess) e = c->Bs.ensure((size_t)(P * c->box[0] * s.w[1] * s.w[2]) * c->csize, c->st);
    return e;
}

// M[a][b][g] = M_{a0+a, b0+b}(k, q, G_g) for bands a0.. at k = kcrys[ik] and
// b0.. at k + q (absolute band indices of the uploads) into the device
// buffer M (row stride ng).  `clean` is cleared when the box aliases.
bgw_status mtxel_into(bgw_ctx_s *c, const char *who, QState &s, int ik, int a0, int na, int b0, int nb2,
                      void *M, bool &clean) {
    int kp, G0[3];
    if (!find_umklapp(c, ik, s.q, kp, G0)) return c->fail(BGW_E_ARG, "%s: k + q is not on the k list (k %d)", who, ik);
    if (!c->k[ik].uploaded || !c->k[kp].uploaded)
        return c->fail(BGW_E_STATE, "%s: k %d or its partner %d not uploaded", who, ik, kp);
    if (na == 0 || nb2 == 0) return BGW_OK;
    clean = clean && alias_free(c, ik, kp, G0, s);
    cudaError_t e = flush_k1(c);
    if (e != cudaSuccess) return c->cuda_fail(e, "deferred sphere-to-grid kernels");
    e = ensure_mtxel_scratch_pairs(c, s, na, nb2);
    if (e != cudaSuccess) return c->cuda_fail(e, "matrix-element scratch");
    e = c->gmap_tmp.ensure(sizeof(int) * s.gmap.size(), c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "map buffer");
    // pageable source: the copy is stream-ordered and has read the host
    // vector when it returns, so the buffer can be refilled by a later call
    e = cudaMemcpyAsync(c->gmap_tmp.p, s.gmap.data(), sizeof(int) * s.gmap.size(), cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "map copy");
    const bgw::Axes ax = mtxel_axes(c, s, G0);
    cudaError_t ge;
    const int sa = ensure_grid(c, ik, ge);
    if (ge != cudaSuccess) return c->cuda_fail(ge, "grid");
    const int sb = ensure_grid(c, kp, ge);
    if (ge != cudaSuccess) return c->cuda_fail(ge, "grid");
    const int *gmap = static_cast<const int *>(c->gmap_tmp.p);
    XProf xp(c);
    e = (c->prec == BGW_FP64)
            ? bgw::mtxel_f64(c->slot_ptr(sa, a0), c->slot_ptr(sb, b0), na, nb2, ax, gmap, s.ng, c->A.p, c->Bs.p, M,
                             s.ng, c->st, 0, 0, c->mtxel_lanes, 0, xp.get())
            : bgw::mtxel_f32(c->slot_ptr(sa, a0), c->slot_ptr(sb, b0), na, nb2, ax, gmap, s.ng, c->A.p, c->Bs.p, M,
                             s.ng, c->st, 0, 0, c->mtxel_lanes, c->mtxel_zy, xp.get(),
                             static_cast<int *>(c->errflag.p));
    xp.finish();
    if (e != cudaSuccess) return c->cuda_fail(e, "matrix-element kernels");
    return BGW_OK;
}

// Grid index j of k - q: the k-point whose k + q lands on kcrys[ik].
int k_minus_q(const bgw_ctx_s *c, int ik, const double q[3]) {
    for (int j = 0; j < c->nk; ++j) {
        int kp, G0[3];
        if (find_umklapp(c, j, q, kp, G0) && kp == ik) return j;
    }
    return -1;
}

}  // namespace

// ---- checkpoint / resume ----------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'B', 'G', 'W', 'C', 'H', 'I', '0', 'K'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t precision;
    uint64_t hash;        // FNV-1a of the problem the sum belongs to
    int32_t nq, nfreq, nk, box0;
    int32_t box1, box2, nv, nc_max;
};
static_assert(sizeof(CkptHeader) == 56, "checkpoint header layout");
static_assert((int)BGW_MIXED_BF16X3 == bgw::kMixedBF16x3 && (int)BGW_MIXED_TF32X3 == bgw::kMixedTF32x3 &&
                  (int)BGW_MIXED_TF32 == bgw::kMixedTF32,
              "mixed operand formats follow bgw_precision");

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
    template <class T> void add(const T &v) { add(&v, sizeof(T)); }
};

// The problem a running sum belongs to: box, k list, band layout, precision,
// q-set (q, sphere, Nc) and frequencies.
uint64_t problem_hash(const bgw_ctx_s *c, const std::vector<QState> &qs, const std::vector<double> &freq) {
    Fnv f;
    f.add(c->box, sizeof(c->box));
    f.add(c->nk);
    f.add(c->kcrys.data(), sizeof(double) * c->kcrys.size());
    f.add(c->nv);
    f.add(c->nc_max);
    f.add((int)c->prec);
    f.add((int)qs.size());
    for (const QState &s : qs) {
        f.add(s.q, sizeof(s.q));
        f.add(s.ng);
        f.add(s.nc);
        f.add(s.gvec.data(), sizeof(int) * s.gvec.size());
    }
    f.add((int)freq.size());
    f.add(freq.data(), sizeof(double) * freq.size());
    return f.h;
}

size_t ckpt_bytes(const bgw_ctx_s *c, const std::vector<QState> &qs, int nfreq) {
    size_t b = sizeof(CkptHeader) + sizeof(int32_t) * (size_t)c->nk;
    b = (b + 15) & ~(size_t)15;
    for (const QState &s : qs) b += 16 + 16 * (size_t)nfreq * s.ng * s.ng;
    return b;
}

}  // namespace

extern "C" {

const char *bgw_version(void) { return "bgwchi 0.1 (sm_103a)"; }

const char *bgw_last_error(bgw_ctx ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

bgw_status bgw_create(bgw_ctx *out, const int fft[3], int nk, const double *kcrys, int nv,
                      int nc_max, bgw_precision prec, void *stream) {
    g_create_error.clear();
    if (!out || !fft || !kcrys) {
        g_create_error = "bgw_create: null pointer argument";
        return BGW_E_ARG;
    }
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (!is_supported_len(fft[a])) {
            g_create_error = "bgw_create: FFT length " + std::to_string(fft[a]) +
                             " not supported (16,18,20,24,27,30,32,36,40,48,64)";
            return BGW_E_ARG;
        }
    if (nk < 1 || nv < 1 || nc_max < 1) {
        g_create_error = "bgw_create: nk, nv and nc_max must be >= 1";
        return BGW_E_ARG;
    }
    if (prec != BGW_FP64 && prec != BGW_MIXED_BF16X3 && prec != BGW_MIXED_TF32X3 && prec != BGW_MIXED_TF32) {
        g_create_error = "bgw_create: unknown precision";
        return BGW_E_ARG;
    }
    for (long i = 0; i < 3L * nk; ++i)
        if (!std::isfinite(kcrys[i])) {
            g_create_error = "bgw_create: non-finite k coordinate";
            return BGW_E_ARG;
        }
    if (const char *f = std::getenv("BGW_FAULT")) {   // BGW_FAULT=oom@n: see g_fail_alloc
        long n = 0;
        if (std::sscanf(f, "oom@%ld", &n) == 1 && n > 0) g_fail_alloc.store(n);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = ensure_tables(dev);
    if (e != cudaSuccess) {
        g_create_error = std::string("bgw_create: ") + cudaGetErrorString(e);
        return BGW_E_CUDA;
    }
    bgw_ctx_s *c = new bgw_ctx_s();
    for (int a = 0; a < 3; ++a) c->box[a] = fft[a];
    c->nbox = (long)fft[0] * fft[1] * fft[2];
    c->nk = nk;
    c->nv = nv;
    c->nc_max = nc_max;
    c->nb = nv + nc_max;
    c->kcrys.assign(kcrys, kcrys + 3L * nk);
    c->prec = prec;
    c->st = static_cast<cudaStream_t>(stream);
    c->device = dev;
    c->csize = (prec == BGW_FP64) ? 16 : 8;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        c->sm_count < 1)
        c->sm_count = 1;
    c->k.resize(nk);
    e = c->energy.ensure(sizeof(double) * (size_t)nk * c->nb, c->st);
    if (e == cudaSuccess) e = c->errflag.ensure(sizeof(int), c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->st);
    if (e != cudaSuccess) {
        g_create_error = std::string("bgw_create: allocating buffers: ") + cudaGetErrorString(e);
        const bgw_status s = (e == cudaErrorMemoryAllocation) ? BGW_E_NOMEM : BGW_E_CUDA;
        cudaGetLastError();
        c->grids.release();
        c->energy.release();
        c->errflag.release();
        delete c;
        return s;
    }
    *out = c;
    return BGW_OK;
}

bgw_status bgw_wfn_upload(bgw_ctx c, int ik, int ngw, const int *gvec, const double *coeff,
                          const double *energy_eV, int on_device) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (ik < 0 || ik >= c->nk) return c->fail(BGW_E_ARG, "wfn_upload: ik=%d outside 0..%d", ik, c->nk - 1);
    if (ngw < 1 || !gvec || !coeff || !energy_eV)
        return c->fail(BGW_E_ARG, "wfn_upload: ngw >= 1 and non-null gvec, coeff, energy required");
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = gvec[a];
    for (long i = 0; i < ngw; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], gvec[3 * i + a]);
            hi[a] = std::max(hi[a], gvec[3 * i + a]);
        }
    int w[3];
    for (int a = 0; a < 3; ++a) {
        w[a] = hi[a] - lo[a] + 1;
        if (w[a] > c->box[a])
            return c->fail(BGW_E_GRID,
                           "wfn_upload: sphere of k %d spans %d points on axis %d, box has %d",
                           ik, w[a], a, c->box[a]);
    }
    std::vector<int> map((size_t)w[0] * w[1] * w[2], -1);
    for (long i = 0; i < ngw; ++i) {
        const long idx = ((long)(gvec[3 * i] - lo[0]) * w[1] + (gvec[3 * i + 1] - lo[1])) * w[2] +
                         (gvec[3 * i + 2] - lo[2]);
        if (map[idx] >= 0)
            return c->fail(BGW_E_ARG, "wfn_upload: duplicate G (%d,%d,%d) in the sphere of k %d",
                           gvec[3 * i], gvec[3 * i + 1], gvec[3 * i + 2], ik);
        map[idx] = (int)i;
    }
    // inverse map (coefficient -> cube cell) after the cube map
    const size_t ncube = map.size();
    map.resize(ncube + ngw);
    for (size_t cell = 0; cell < ncube; ++cell)
        if (map[cell] >= 0) map[ncube + map[cell]] = (int)cell;
    const long B = 2L * c->nb;
    cudaError_t e;
    KPoint &kp = c->k[ik];
    // device copy of the cube map (only when it changed)
    const bool map_changed = kp.cube_map != map;
    if (map_changed) {
        e = kp.map_dev.ensure(sizeof(int) * map.size(), c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: map buffer");
        kp.cube_map.swap(map);
        e = cudaMemcpyAsync(kp.map_dev.p, kp.cube_map.data(), sizeof(int) * kp.cube_map.size(),
                            cudaMemcpyHostToDevice, c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: map copy");
    }
    e = ensure_slots(c);
    if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: real-space grids");
    const size_t cbytes = sizeof(double) * 2 * (size_t)B * ngw;
    const double *src = coeff;
    if (c->streaming()) {
        // keep the coefficients (device inputs by reference, host inputs in a
        // device copy); the grid is built when a k-chunk needs it
        if (on_device) {
            kp.coeff.release();
            kp.coeff_src = coeff;
        } else {
            e = kp.coeff.ensure(cbytes, c->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(kp.coeff.p, coeff, cbytes, cudaMemcpyHostToDevice, c->st);
            if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: coefficient store");
            kp.coeff_src = static_cast<const double *>(kp.coeff.p);
        }
    } else if (c->copy_ahead && !on_device && !st_capturing(c)) {
        // copy on the copy stream into the k's own buffer, once the last
        // transform that read that buffer has run; the transform waits for it
        e = ensure_copy_events(c, kp);
        if (e == cudaSuccess && !kp.consumed_set) {
            // first copy-ahead copy of this k: after everything queued so far
            e = cudaEventRecord(kp.consumed, c->st);
            kp.consumed_set = true;
        }
        cudaStream_t cs = c->cst[ik % bgw_ctx_s::kCopyStreams];
        if (e == cudaSuccess && cbytes > kp.coeff.cap) e = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = kp.coeff.ensure(cbytes, c->st);
        if (e == cudaSuccess && kp.consumed_set) e = cudaStreamWaitEvent(cs, kp.consumed, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(kp.coeff.p, coeff, cbytes, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(kp.copied, cs);
        // the k's transform waits for the copy: a deferred build (flush_k1)
        // adds that wait just before it, so the copy can run beside the work
        // already queued on the context stream; an immediate build waits here
        if (c->defer_k1)
            kp.copy_wait = true;
        else if (e == cudaSuccess)
            e = cudaStreamWaitEvent(c->st, kp.copied, 0);
        if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: copy-ahead coefficient copy");
        src = static_cast<const double *>(kp.coeff.p);
    } else if (c->defer_k1) {
        // the grid is built by the next call that reads grids; host inputs
        // are kept in a per-k device copy until then
        if (!on_device) {
            e = kp.coeff.ensure(cbytes, c->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(kp.coeff.p, coeff, cbytes, cudaMemcpyHostToDevice, c->st);
            if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: coefficient store");
            src = static_cast<const double *>(kp.coeff.p);
        }
    } else if (!on_device) {
        e = c->stage.ensure(cbytes, c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: staging buffer");
        e = cudaMemcpyAsync(c->stage.p, coeff, cbytes, cudaMemcpyHostToDevice, c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: coefficient copy");
        src = static_cast<const double *>(c->stage.p);
    }
    e = cudaMemcpyAsync(static_cast<double *>(c->energy.p) + (long)ik * c->nb, energy_eV,
                        sizeof(double) * c->nb,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: energy copy");
    for (int a = 0; a < 3; ++a) {
        kp.lo[a] = lo[a];
        kp.hi[a] = hi[a];
    }
    kp.ngw = ngw;
    if (c->streaming()) {
        if (kp.slot >= 0) {            // the cached grid is stale now
            c->slot_k[kp.slot] = -1;
            c->slot_stamp[kp.slot] = 0;
            kp.slot = -1;
        }
    } else if (c->defer_k1) {
        if (!kp.pending) ++c->npending;
        kp.pending = src;
    } else {
        if (kp.pending) {                // a deferred build of an older upload is void now
            kp.pending = nullptr;
            --c->npending;
        }
        e = run_k1(c, ik, src, ik);
        if (e == cudaSuccess && src == kp.coeff.p) e = mark_consumed(c, kp);
        if (e != cudaSuccess) return c->cuda_fail(e, "wfn_upload: sphere-to-grid kernels");
    }
    kp.uploaded = true;
    return BGW_OK;
}

bgw_status bgw_mtxel_spinor(bgw_ctx c, const bgw_q *q, int ik, int v0, int nv, int c0, int nc,
                            void *M_dev) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!M_dev) return c->fail(BGW_E_ARG, "mtxel: null output");
    if (ik < 0 || ik >= c->nk) return c->fail(BGW_E_ARG, "mtxel: ik=%d out of range", ik);
    if (nv < 0 || v0 < 0 || v0 + nv > c->nv) return c->fail(BGW_E_ARG, "mtxel: valence range");
    if (nc < 0 || c0 < 0 || c0 + nc > c->nc_max) return c->fail(BGW_E_ARG, "mtxel: conduction range");
    QState s;
    bgw_status st = prepare_q(c, q, s);
    if (st != BGW_OK) return st;
    int kp, G0[3];
    if (!find_umklapp(c, ik, s.q, kp, G0))
        return c->fail(BGW_E_ARG, "mtxel: k + q is not on the k list (k %d)", ik);
    if (!c->k[ik].uploaded || !c->k[kp].uploaded)
        return c->fail(BGW_E_STATE, "mtxel: k %d or its partner %d not uploaded", ik, kp);
    if (nv == 0 || nc == 0) return BGW_OK;
    const bool clean = alias_free(c, ik, kp, G0, s);
    const long P = (long)nv * nc;
    cudaError_t e = flush_k1(c);
    if (e != cudaSuccess) return c->cuda_fail(e, "mtxel: deferred sphere-to-grid kernels");
    e = ensure_mtxel_scratch(c, s, P);
    if (e != cudaSuccess) return c->cuda_fail(e, "mtxel: scratch");
    // The per-call map goes to a context buffer; reuse is stream-ordered and
    // a pageable-memory copy has read the host vector when the call returns.
    e = c->gmap_tmp.ensure(sizeof(int) * s.gmap.size(), c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "mtxel: map buffer");
    e = cudaMemcpyAsync(c->gmap_tmp.p, s.gmap.data(), sizeof(int) * s.gmap.size(), cudaMemcpyHostToDevice,
                        c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "mtxel: map copy");
    s.gmap_dev.p = c->gmap_tmp.p;   // borrowed, not owned
    e = launch_mtxel(c, s, ik, kp, G0, v0, nv, c0, nc, M_dev, s.ng);
    s.gmap_dev.p = nullptr;
    if (e != cudaSuccess) return c->cuda_fail(e, "mtxel: kernels");
    return clean ? BGW_OK : BGW_W_ALIAS;
}

bgw_status bgw_chi0_reset(bgw_ctx c) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    // The buffers stay allocated for reuse by the next q-set of the same
    // shapes; the next accumulate zeroes them on the stream.  No host sync.
    c->have_qset = false;
    return BGW_OK;
}

bgw_status bgw_chi0_accumulate(bgw_ctx c, int nq, const bgw_q *qs, int nfreq,
                               const double *freq_eV, int k_begin, int k_end) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    std::vector<QState> fresh;
    bgw_status vst = validate_qset(c, "accumulate", nq, qs, nfreq, freq_eV, k_begin, k_end, fresh);
    if (vst != BGW_OK) return vst;
    if (c->have_qset) {
        bool same = (int)c->qs.size() == nq && c->nfreq == nfreq &&
                    std::equal(c->freq.begin(), c->freq.end(), freq_eV);
        for (int iq = 0; same && iq < nq; ++iq) same = same_q(c->qs[iq], &qs[iq]);
        if (!same)
            return c->fail(BGW_E_STATE,
                           "accumulate: q-set or frequencies differ from the running sum; call bgw_chi0_reset");
    }
    const int kchunk = std::max(1, std::min(c->kchunk, std::max(1, k_end - k_begin)));
    cudaError_t e = ensure_chunk_scratch(c, fresh, nfreq, kchunk);
    if (e != cudaSuccess) return c->cuda_fail(e, "accumulate: scratch");
    if (!c->have_qset) {
        bgw_status st = install_qset(c, fresh, nfreq, freq_eV);
        if (st != BGW_OK) return st;
    }
    e = flush_k1(c);
    if (e != cudaSuccess) return c->cuda_fail(e, "accumulate: deferred sphere-to-grid kernels");
    bool clean = true;
    e = run_range(c, c->qs, nfreq, static_cast<const double *>(c->freq_dev.p), k_begin, k_end, kchunk,
                  c->tile_v, c->tile_c, clean);
    if (e != cudaSuccess) return c->cuda_fail(e, "accumulate: kernels");
    for (int k = k_begin; k < k_end; ++k) ++c->kcount[k];
    return clean ? BGW_OK : BGW_W_ALIAS;
}

bgw_status bgw_chi0_finalize(bgw_ctx c, int iq, void *chi0, int on_device) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!chi0) return c->fail(BGW_E_ARG, "finalize: null output");
    if (!c->have_qset) return c->fail(BGW_E_STATE, "finalize: nothing accumulated");
    if (iq < 0 || iq >= (int)c->qs.size()) return c->fail(BGW_E_ARG, "finalize: iq=%d out of range", iq);
    QState &s = c->qs[iq];
    const size_t bytes = 16 * (size_t)c->nfreq * s.ng * s.ng;
    const double scale = 1.0 / c->nk;
    cudaError_t e;
    if (on_device) {
        const int rec = c->stage_begin(4);
        e = bgw::chi0_finalize(s.acc.p, s.ng, c->nfreq, scale, chi0, c->st);
        c->stage_end(rec, 1);
        if (e != cudaSuccess) return c->cuda_fail(e, "finalize: kernel");
        return BGW_OK;
    }
    e = c->out_stage.ensure(bytes, c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "finalize: staging");
    const int rec = c->stage_begin(4);
    e = bgw::chi0_finalize(s.acc.p, s.ng, c->nfreq, scale, c->out_stage.p, c->st);
    c->stage_end(rec, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(chi0, c->out_stage.p, bytes, cudaMemcpyDeviceToHost, c->st);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "finalize: copy to host");
    if (flag == bgw::F64TC_ERR_SIGN) {
        cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->st);
        return c->fail(BGW_E_ARG, "finalize: a pair weight was positive (an occupied band above an empty one); "
                                  "the tensor-core FP64 contraction needs every e_v < e_c: set "
                                  "BGW_OPT_FP64_CONTRACTION to 1 for such inputs");
    }
    if (flag != 0) {
        cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->st);
        return c->fail(BGW_E_TIMEOUT, "finalize: a device-side wait gave up (code %d); the result is invalid",
                       flag);
    }
    return BGW_OK;
}

// ---- checkpoint / resume (format and problem hash defined before extern "C") ----

bgw_status bgw_chi0_progress(bgw_ctx c, int *k_counts) {
    if (!c) return BGW_E_ARG;
    c->err.clear();
    if (!k_counts) return c->fail(BGW_E_ARG, "progress: null output");
    if (!c->have_qset) return c->fail(BGW_E_STATE, "progress: no running sum");
    std::copy(c->kcount.begin(), c->kcount.end(), k_counts);
    return BGW_OK;
}

bgw_status bgw_chi0_checkpoint_bytes(bgw_ctx c, size_t *bytes) {
    if (!c) return BGW_E_ARG;
    c->err.clear();
    if (!bytes) return c->fail(BGW_E_ARG, "checkpoint_bytes: null output");
    if (!c->have_qset) return c->fail(BGW_E_STATE, "checkpoint_bytes: no running sum");
    *bytes = ckpt_bytes(c, c->qs, c->nfreq);
    return BGW_OK;
}

bgw_status bgw_chi0_checkpoint(bgw_ctx c, void *buf, size_t bytes) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!buf) return c->fail(BGW_E_ARG, "checkpoint: null buffer");
    if (!c->have_qset) return c->fail(BGW_E_STATE, "checkpoint: no running sum");
    if (c->capturing) return c->fail(BGW_E_STATE, "checkpoint: not allowed during graph capture");
    const size_t need = ckpt_bytes(c, c->qs, c->nfreq);
    if (bytes < need) return c->fail(BGW_E_ARG, "checkpoint: buffer of %zu bytes, %zu needed", bytes, need);
    char *o = static_cast<char *>(buf);
    CkptHeader h;
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.precision = (uint32_t)c->prec;
    h.hash = problem_hash(c, c->qs, c->freq);
    h.nq = (int32_t)c->qs.size();
    h.nfreq = c->nfreq;
    h.nk = c->nk;
    h.box0 = c->box[0];
    h.box1 = c->box[1];
    h.box2 = c->box[2];
    h.nv = c->nv;
    h.nc_max = c->nc_max;
    std::memcpy(o, &h, sizeof(h));
    std::memcpy(o + sizeof(h), c->kcount.data(), sizeof(int32_t) * (size_t)c->nk);
    size_t off = (sizeof(h) + sizeof(int32_t) * (size_t)c->nk + 15) & ~(size_t)15;
    cudaError_t e = cudaSuccess;
    for (const QState &s : c->qs) {
        const int32_t hdr[4] = {s.ng, s.nc, 0, 0};
        std::memcpy(o + off, hdr, sizeof(hdr));
        off += 16;
        const size_t ab = 16 * (size_t)c->nfreq * s.ng * s.ng;
        if (e == cudaSuccess) e = cudaMemcpyAsync(o + off, s.acc.p, ab, cudaMemcpyDeviceToHost, c->st);
        off += ab;
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "checkpoint: copy to host");
    if (flag == bgw::F64TC_ERR_SIGN)
        return c->fail(BGW_E_ARG, "checkpoint: a pair weight was positive; the tensor-core FP64 contraction "
                                  "left it out (set BGW_OPT_FP64_CONTRACTION to 1 for such inputs)");
    if (flag != 0)
        return c->fail(BGW_E_TIMEOUT, "checkpoint: a device-side wait gave up (code %d); the sum is invalid", flag);
    return BGW_OK;
}

bgw_status bgw_chi0_resume(bgw_ctx c, int nq, const bgw_q *qs, int nfreq, const double *freq_eV,
                           const void *buf, size_t bytes) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!buf) return c->fail(BGW_E_ARG, "resume: null buffer");
    if (c->capturing) return c->fail(BGW_E_STATE, "resume: not allowed during graph capture");
    std::vector<QState> fresh;
    bgw_status vst = validate_qset(c, "resume", nq, qs, nfreq, freq_eV, 0, 0, fresh);
    if (vst != BGW_OK) return vst;
    const size_t need = ckpt_bytes(c, fresh, nfreq);
    const char *in = static_cast<const char *>(buf);
    CkptHeader h;
    if (bytes < sizeof(h)) return c->fail(BGW_E_ARG, "resume: buffer too small for a checkpoint");
    std::memcpy(&h, in, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion)
        return c->fail(BGW_E_ARG, "resume: not a checkpoint of this format");
    std::vector<double> fv(freq_eV, freq_eV + nfreq);
    if (h.hash != problem_hash(c, fresh, fv) || h.nq != nq || h.nfreq != nfreq || h.nk != c->nk)
        return c->fail(BGW_E_STATE, "resume: the checkpoint belongs to another problem or q-set");
    if (bytes < need) return c->fail(BGW_E_ARG, "resume: buffer of %zu bytes, %zu needed", bytes, need);
    c->have_qset = false;
    bgw_status st = install_qset(c, fresh, nfreq, freq_eV);   // zeroes the accumulators on the stream
    if (st != BGW_OK) return st;
    std::memcpy(c->kcount.data(), in + sizeof(h), sizeof(int32_t) * (size_t)c->nk);
    size_t off = (sizeof(h) + sizeof(int32_t) * (size_t)c->nk + 15) & ~(size_t)15;
    cudaError_t e = cudaSuccess;
    for (QState &s : c->qs) {
        off += 16;
        const size_t ab = 16 * (size_t)nfreq * s.ng * s.ng;
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.acc.p, in + off, ab, cudaMemcpyHostToDevice, c->st);
        off += ab;
    }
    // pageable source: wait so the caller may free or reuse the buffer at once
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        c->have_qset = false;
        return c->cuda_fail(e, "resume: copy to device");
    }
    return BGW_OK;
}

bgw_status bgw_set_option(bgw_ctx c, int option, long value) {
    if (!c) return BGW_E_ARG;
    c->err.clear();
    switch (option) {
        case BGW_OPT_KCHUNK:
            if (value < 1 || value > 256) return c->fail(BGW_E_ARG, "set_option: k-chunk must be 1..256");
            c->kchunk = (int)value;
            return BGW_OK;
        case BGW_OPT_PAIR_TILE_V:
        case BGW_OPT_PAIR_TILE_C:
            if (value < 0 || value > 16) return c->fail(BGW_E_ARG, "set_option: pair tile must be 0..16");
            (option == BGW_OPT_PAIR_TILE_V ? c->tile_v : c->tile_c) = (int)value;
            return BGW_OK;
        case BGW_OPT_TEST_DROP_LOAD:
            if (value < 0 || value > 2) return c->fail(BGW_E_ARG, "set_option: test drop load must be 0, 1 or 2");
            c->test_drop_load = (int)value;
            return BGW_OK;
        case BGW_OPT_K1_PATH:
            if (value < 0 || value > 4) return c->fail(BGW_E_ARG, "set_option: K1 path must be 0..4");
            c->k1_path = (int)value;
            return BGW_OK;
        case BGW_OPT_MTXEL_LANES:
            if (value != 0 && value != 1 && value != 8)
                return c->fail(BGW_E_ARG, "set_option: matrix-element lanes must be 0, 1 or 8");
            c->mtxel_lanes = (int)value;
            return BGW_OK;
        case BGW_OPT_DEFER_K1:
            if (value != 0 && value != 1) return c->fail(BGW_E_ARG, "set_option: deferred K1 must be 0 or 1");
            c->defer_k1 = (int)value;
            return BGW_OK;
        case BGW_OPT_COPY_AHEAD:
            if (value != 0 && value != 1) return c->fail(BGW_E_ARG, "set_option: copy-ahead must be 0 or 1");
            c->copy_ahead = (int)value;
            return BGW_OK;
        case BGW_OPT_OVERLAP:
            if (value != 0 && value != 1) return c->fail(BGW_E_ARG, "set_option: overlap must be 0 or 1");
            if (c->capturing) return c->fail(BGW_E_STATE, "set_option: overlap cannot change during a capture");
            c->overlap = (int)value;
            return BGW_OK;
        case BGW_OPT_MTXEL_ZY:
            if (value < 0 || value > 2) return c->fail(BGW_E_ARG, "set_option: matrix-element z+y kernel must be 0, 1 or 2");
            c->mtxel_zy = (int)value;
            return BGW_OK;
        case BGW_OPT_FP64_CONTRACTION:
            if (value != 0 && value != 1) return c->fail(BGW_E_ARG, "set_option: FP64 contraction must be 0 or 1");
            if (c->capturing) return c->fail(BGW_E_STATE, "set_option: contraction kernel cannot change during a capture");
            c->f64_dfma = (int)value;
            return BGW_OK;
        case BGW_OPT_TEST_FAIL_ALLOC:
            if (value < 0) return c->fail(BGW_E_ARG, "set_option: allocation count must be >= 0");
            g_fail_alloc.store(value);
            return BGW_OK;
        case BGW_OPT_GRID_SLOTS:
            if (c->nslots > 0) return c->fail(BGW_E_STATE, "set_option: grid slots are fixed at the first upload");
            if (value < 0 || value > c->nk) return c->fail(BGW_E_ARG, "set_option: grid slots must be 0..nk");
            c->grid_slots_opt = (int)value;
            return BGW_OK;
        default:
            return c->fail(BGW_E_ARG, "set_option: unknown option %d", option);
    }
}

bgw_status bgw_get_option(bgw_ctx c, int option, long *value) {
    if (!c || !value) return BGW_E_ARG;
    c->err.clear();
    switch (option) {
        case BGW_OPT_KCHUNK: *value = c->kchunk; return BGW_OK;
        case BGW_OPT_PAIR_TILE_V: *value = c->tile_v; return BGW_OK;
        case BGW_OPT_PAIR_TILE_C: *value = c->tile_c; return BGW_OK;
        case BGW_OPT_GRID_SLOTS: *value = c->nslots > 0 ? c->nslots : c->grid_slots_opt; return BGW_OK;
        case BGW_OPT_TEST_DROP_LOAD: *value = c->test_drop_load; return BGW_OK;
        case BGW_OPT_TEST_FAIL_ALLOC: *value = g_fail_alloc.load(); return BGW_OK;
        case BGW_OPT_K1_PATH: *value = c->k1_path; return BGW_OK;
        case BGW_OPT_MTXEL_LANES: *value = c->mtxel_lanes; return BGW_OK;
        case BGW_OPT_DEFER_K1: *value = c->defer_k1; return BGW_OK;
        case BGW_OPT_COPY_AHEAD: *value = c->copy_ahead; return BGW_OK;
        case BGW_OPT_OVERLAP: *value = c->overlap; return BGW_OK;
        case BGW_OPT_FP64_CONTRACTION: *value = c->f64_dfma; return BGW_OK;
        case BGW_OPT_MTXEL_ZY: *value = c->mtxel_zy; return BGW_OK;
        default: return c->fail(BGW_E_ARG, "get_option: unknown option %d", option);
    }
}

bgw_status bgw_autotune(bgw_ctx c, int nq, const bgw_q *qs, int nfreq, const double *freq_eV,
                        int k_begin, int k_end, const char *cache_path) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    std::vector<QState> tq;
    bgw_status vst = validate_qset(c, "autotune", nq, qs, nfreq, freq_eV, k_begin, k_end, tq);
    if (vst != BGW_OK) return vst;
    if (k_end == k_begin) return c->fail(BGW_E_ARG, "autotune: empty k range");
    // cache key: everything the timing depends on
    static const char *const prec_name[] = {"fp64", "mixed", "tf32x3", "tf32"};
    std::string key = std::string(prec_name[c->prec]) + " box " +
                      std::to_string(c->box[0]) + "x" + std::to_string(c->box[1]) + "x" +
                      std::to_string(c->box[2]) + " nv " + std::to_string(c->nv) + " nfreq " +
                      std::to_string(nfreq) + " span " + std::to_string(k_end - k_begin);
    for (auto &s : tq) key += " q " + std::to_string(s.ng) + "/" + std::to_string(s.nc);
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "r")) {
            char line[1024];
            while (fgets(line, sizeof line, f)) {
                const char *bar = strchr(line, '|');
                if (!bar || std::string(line, bar - line) != key) continue;
                int kc, tv, tcc, zy = 0;
                const int got = sscanf(bar + 1, "%d %d %d %d", &kc, &tv, &tcc, &zy);
                if (got >= 3) {
                    c->kchunk = kc;
                    c->tile_v = tv;
                    c->tile_c = tcc;
                    if (got == 4) c->mtxel_zy = zy;
                    fclose(f);
                    return BGW_OK;
                }
            }
            fclose(f);
        }
    }
    // scratch accumulators and maps for the timing runs (the running sums are untouched)
    cudaError_t e = flush_k1(c);
    if (e != cudaSuccess) return c->cuda_fail(e, "autotune: deferred sphere-to-grid kernels");
    const bool prof = c->prof;
    c->prof = false;
    DevBuf tfreq;
    e = tfreq.ensure(sizeof(double) * nfreq, c->st);
    for (auto &s : tq) {
        if (e == cudaSuccess) e = s.gmap_dev.ensure(sizeof(int) * s.gmap.size(), c->st);
        if (e == cudaSuccess) e = s.kmap_dev.ensure(sizeof(int) * (size_t)c->nk, c->st);
        if (e == cudaSuccess) e = s.acc.ensure(16 * (size_t)nfreq * s.ng * s.ng, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.gmap_dev.p, s.gmap.data(), sizeof(int) * s.gmap.size(),
                                                  cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.kmap_dev.p, s.kmap.data(), sizeof(int) * c->nk,
                                                  cudaMemcpyHostToDevice, c->st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tfreq.p, freq_eV, sizeof(double) * nfreq, cudaMemcpyHostToDevice, c->st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    long Pmax = 0;
    for (auto &s : tq) Pmax = std::max(Pmax, (long)c->nv * s.nc);
    // one warm-up run, then the median of three timed runs
    auto time_one = [&](int kc, int tv, int tcc, float &ms) -> cudaError_t {
        cudaError_t r = ensure_chunk_scratch(c, tq, nfreq, kc);
        bool clean = true;
        const double *fq = static_cast<const double *>(tfreq.p);
        if (r == cudaSuccess) r = run_range(c, tq, nfreq, fq, k_begin, k_end, kc, tv, tcc, clean);   // warm
        float t[3] = {0, 0, 0};
        for (int i = 0; i < 3 && r == cudaSuccess; ++i) {
            r = cudaEventRecord(e0, c->st);
            if (r == cudaSuccess) r = run_range(c, tq, nfreq, fq, k_begin, k_end, kc, tv, tcc, clean);
            if (r == cudaSuccess) r = cudaEventRecord(e1, c->st);
            if (r == cudaSuccess) r = cudaEventSynchronize(e1);
            if (r == cudaSuccess) r = cudaEventElapsedTime(&t[i], e0, e1);
        }
        std::sort(t, t + 3);
        ms = t[1];
        return r;
    };
    const int zy_in = c->mtxel_zy;
    int best_kc = c->kchunk, best_tv = c->tile_v, best_tc = c->tile_c, best_zy = zy_in;
    float best_ms = 1e30f;
    if (e == cudaSuccess) {
        // matrix-element kernel first (FP32: the streamed z + y kernel and the
        // plane kernel's best pair tiles), at k-chunk 1
        int tvs[8] = {0}, tcs[8] = {0}, zys[8] = {zy_in};
        int ncand = 1;
        if (c->prec != BGW_FP64) {
            const int zero3[3] = {0, 0, 0};
            bgw::Axes ax = mtxel_axes(c, tq[0], zero3);
            zys[0] = 2;
            const int nt = bgw::plane_tile_candidates(c->nv, tq[0].nc, ax, tvs + 1, tcs + 1, 4);
            for (int i = 1; i <= nt; ++i) zys[i] = 1;
            ncand += nt;
        }
        for (int i = 0; i < ncand && e == cudaSuccess; ++i) {
            float ms = 0;
            c->mtxel_zy = zys[i];
            e = time_one(1, tvs[i], tcs[i], ms);
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best_tv = tvs[i];
                best_tc = tcs[i];
                best_zy = zys[i];
                best_kc = 1;
            }
        }
        c->mtxel_zy = best_zy;
        // then the k-chunk, within a workspace cap (the split operands of the
        // mixed path grow with the chunk)
        const int kcands[] = {2, 4, 8, 16, 32, 64};
        for (int kc : kcands) {
            if (e != cudaSuccess || kc > k_end - k_begin) break;
            size_t ws = 0, mb = 0;
            for (auto &s : tq) {
                mb = std::max(mb, (size_t)kc * c->nv * s.nc * s.ng * c->csize);
                if (c->prec != BGW_FP64)
                    ws = std::max(ws, bgw::mixed_workspace_bytes((long)kc * c->nv * s.nc, s.ng, nfreq, (int)c->prec));
                else
                    ws = std::max(ws, f64_ws_bytes(c, (long)kc * c->nv * s.nc, s.ng, nfreq));
            }
            if (ws + mb > ((size_t)2 << 30)) break;
            float ms = 0;
            e = time_one(kc, best_tv, best_tc, ms);
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best_kc = kc;
            }
        }
    }
    cudaStreamSynchronize(c->st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    tfreq.release();
    for (auto &s : tq) {
        s.gmap_dev.release();
        s.kmap_dev.release();
        s.acc.release();
    }
    c->prof = prof;
    if (e != cudaSuccess) {
        c->mtxel_zy = zy_in;
        return c->cuda_fail(e, "autotune");
    }
    c->kchunk = best_kc;
    c->tile_v = best_tv;
    c->tile_c = best_tc;
    c->mtxel_zy = best_zy;
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "a")) {
            fprintf(f, "%s|%d %d %d %d\n", key.c_str(), best_kc, best_tv, best_tc, best_zy);
            fclose(f);
        }
    }
    return BGW_OK;
}

bgw_status bgw_graph_begin(bgw_ctx c) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!c->st) return c->fail(BGW_E_ARG, "graph_begin: the context stream is the legacy default stream");
    if (c->capturing) return c->fail(BGW_E_STATE, "graph_begin: already capturing");
    cudaError_t e = flush_k1(c);   // uploads made before the capture are not part of it
    if (e == cudaSuccess) e = c->drain();
    for (int i = 0; i < bgw_ctx_s::kCopyStreams && e == cudaSuccess; ++i)
        if (c->cst[i]) e = cudaStreamSynchronize(c->cst[i]);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return c->cuda_fail(e, "graph_begin");
    c->capturing = true;
    return BGW_OK;
}

bgw_status bgw_graph_end(bgw_ctx c) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!c->capturing) return c->fail(BGW_E_STATE, "graph_end: not capturing");
    c->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->st, &g);
    if (e != cudaSuccess || !g) {
        cudaGetLastError();
        return c->cuda_fail(e != cudaSuccess ? e : cudaErrorStreamCaptureInvalidated, "graph_end");
    }
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        return c->cuda_fail(e, "graph_end: instantiate");
    }
    return BGW_OK;
}

bgw_status bgw_graph_launch(bgw_ctx c) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!c->gexec) return c->fail(BGW_E_STATE, "graph_launch: nothing captured");
    if (c->capturing) return c->fail(BGW_E_STATE, "graph_launch: still capturing");
    cudaError_t e = cudaGraphLaunch(c->gexec, c->st);
    // the graph may read any k's copy-ahead buffer
    for (auto &kp : c->k)
        if (e == cudaSuccess && kp.consumed) {
            e = cudaEventRecord(kp.consumed, c->st);
            kp.consumed_set = true;
        }
    if (e != cudaSuccess) return c->cuda_fail(e, "graph_launch");
    return BGW_OK;
}

bgw_status bgw_profile(bgw_ctx c, int enable) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    cudaError_t e = c->drain();
    if (e != cudaSuccess) return c->cuda_fail(e, "profile: stream");
    if (enable) {
        for (int i = 0; i < bgw_ctx_s::kStages; ++i) {
            c->prof_ms[i] = 0;
            c->prof_calls[i] = c->prof_kernels[i] = 0;
        }
    }
    c->prof = enable != 0;
    return BGW_OK;
}

bgw_status bgw_profile_read(bgw_ctx c, double *ms, long *calls, long *kernels, int n) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (c->capturing) return c->fail(BGW_E_STATE, "profile_read: not allowed during graph capture");
    if (n < 0 || n > bgw_ctx_s::kStages) return c->fail(BGW_E_ARG, "profile_read: n outside 0..7");
    cudaError_t e = c->drain();
    if (e != cudaSuccess) return c->cuda_fail(e, "profile_read: stream");
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = c->prof_ms[i];
        if (calls) calls[i] = c->prof_calls[i];
        if (kernels) kernels[i] = c->prof_kernels[i];
    }
    return BGW_OK;
}

void bgw_destroy(bgw_ctx c) {
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        if (c->capturing) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->st, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
        cudaStreamSynchronize(c->st);
        for (cudaStream_t cs : c->cst)
            if (cs) {
                cudaStreamSynchronize(cs);
                cudaStreamDestroy(cs);
            }
        if (c->gst) {
            cudaStreamSynchronize(c->gst);
            cudaStreamDestroy(c->gst);
        }
        for (cudaEvent_t ev : {c->ov_fork, c->ov_join, c->ov_free[0], c->ov_free[1]})
            if (ev) cudaEventDestroy(ev);
        for (auto &k : c->k) {
            if (k.copied) cudaEventDestroy(k.copied);
            if (k.consumed) cudaEventDestroy(k.consumed);
        }
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        for (auto &r : c->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto ev : c->pool) cudaEventDestroy(ev);
        for (auto &k : c->k) {
            k.map_dev.release();
            k.coeff.release();
        }
        for (auto &s : c->qs) {
            s.gmap_dev.release();
            s.kmap_dev.release();
            s.acc.release();
        }
        DevBuf *bufs[] = {&c->grids, &c->energy, &c->stage, &c->S,  &c->R,        &c->A,
                          &c->Bs,    &c->M,      &c->W,     &c->mixed_ws, &c->freq_dev, &c->out_stage, &c->gmap_tmp,
                          &c->errflag, &c->nx_m1, &c->nx_m2, &c->nx_y, &c->nx_t, &c->nx_s, &c->nx_v};
        for (DevBuf *b : bufs) b->release();
    }
    delete c;
}

bgw_status bgw_bounds_check(unsigned *word) {
    if (!word) {
        bgw_set_global_error("bounds_check: null pointer argument");
        return BGW_E_ARG;
    }
    *word = 0u;
    if (!bgw::kBoundsBuild) {
        bgw_set_global_error("bounds_check: this library was built without BGW_BOUNDS (no index checks)");
        return BGW_E_STATE;
    }
    unsigned a = 0u, b = 0u, d = 0u;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = bgw::bounds_take_grid_f64(&a);
    if (e == cudaSuccess) e = bgw::bounds_take_grid_f32(&b);
    if (e == cudaSuccess) e = bgw::bounds_take_chi0(&d);
    if (e != cudaSuccess) {
        bgw_set_global_error(std::string("bounds_check: ") + cudaGetErrorString(e));
        return BGW_E_CUDA;
    }
    *word = a | b | d;
    return BGW_OK;
}

bgw_status bgw_mtxel_bands(bgw_ctx c, const bgw_q *q, int ik, int n0, int nn, int m0, int nm, void *M_dev) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (!M_dev) return c->fail(BGW_E_ARG, "mtxel_bands: null output");
    if (ik < 0 || ik >= c->nk) return c->fail(BGW_E_ARG, "mtxel_bands: ik=%d out of range", ik);
    if (nn < 0 || n0 < 0 || n0 + nn > c->nb || nm < 0 || m0 < 0 || m0 + nm > c->nb)
        return c->fail(BGW_E_ARG, "mtxel_bands: band ranges [%d,%d) and [%d,%d) must lie in [0,%d)", n0, n0 + nn,
                       m0, m0 + nm, c->nb);
    QState s;
    bgw_status st = prepare_q(c, q, s, false);
    if (st != BGW_OK) return st;
    bool clean = true;
    st = mtxel_into(c, "mtxel_bands", s, ik, n0, nn, m0, nm, M_dev, clean);
    if (st != BGW_OK) return st;
    return clean ? BGW_OK : BGW_W_ALIAS;
}

bgw_status bgw_sigma_cohsex(bgw_ctx c, const bgw_q *q, int ik, int n0, int nn, const void *W_dev,
                            const double *vq, double *sx, double *coh) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (c->prec != BGW_FP64) return c->fail(BGW_E_STATE, "sigma_cohsex: needs a BGW_FP64 context");
    if (!W_dev || !vq || !sx || !coh) return c->fail(BGW_E_ARG, "sigma_cohsex: null pointer argument");
    if (ik < 0 || ik >= c->nk) return c->fail(BGW_E_ARG, "sigma_cohsex: ik=%d out of range", ik);
    if (nn < 1 || n0 < 0 || n0 + nn > c->nb)
        return c->fail(BGW_E_ARG, "sigma_cohsex: band range [%d,%d) outside [0,%d)", n0, n0 + nn, c->nb);
    if (st_capturing(c)) return c->fail(BGW_E_STATE, "sigma_cohsex: blocks on its result, cannot be captured");
    QState s;
    bgw_status st = prepare_q(c, q, s, false);
    if (st != BGW_OK) return st;
    for (int g = 0; g < s.ng; ++g)
        if (!std::isfinite(vq[g]) || vq[g] < 0) return c->fail(BGW_E_ARG, "sigma_cohsex: v(q+G) must be finite, >= 0");
    const int jk = k_minus_q(c, ik, s.q);
    if (jk < 0) return c->fail(BGW_E_ARG, "sigma_cohsex: k - q is not on the k list (k %d)", ik);
    const long P = (long)c->nb * nn;
    const size_t mb = 16 * (size_t)P * s.ng;
    cudaError_t e = c->nx_m1.ensure(mb, c->st);
    if (e == cudaSuccess) e = c->nx_y.ensure(mb, c->st);
    if (e == cudaSuccess) e = c->nx_s.ensure(sizeof(double) * (2 * (size_t)P + 3 * (size_t)nn), c->st);
    if (e == cudaSuccess) e = c->nx_v.ensure(sizeof(double) * (size_t)s.ng, c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "sigma_cohsex: scratch");
    // M_{n'' n}(k - q, q, G): every band n'' at k - q, bands n0.. at k
    bool clean = true;
    st = mtxel_into(c, "sigma_cohsex", s, jk, 0, c->nb, n0, nn, c->nx_m1.p, clean);
    if (st != BGW_OK) return st;
    double *sw = static_cast<double *>(c->nx_s.p), *tv = sw + P, *out = tv + P;
    e = cudaMemcpyAsync(c->nx_v.p, vq, sizeof(double) * s.ng, cudaMemcpyHostToDevice, c->st);
    // Y[p][G] = sum_G' W[G][G'] M[p][G']
    if (e == cudaSuccess)
        e = bgw::zgemm_f64((int)P, s.ng, s.ng, c->nx_m1.p, s.ng, 1, false, W_dev, 1, s.ng, false, nullptr, c->nx_y.p,
                           s.ng, 1, 1.0, 0.0, false, c->st);
    if (e == cudaSuccess)
        e = bgw::rowdot_f64(c->nx_m1.p, c->nx_y.p, static_cast<const double *>(c->nx_v.p), P, s.ng, sw, tv, c->st);
    if (e == cudaSuccess) e = bgw::band_sum_f64(sw, c->nv, nn, out, c->st);              // occupied n''
    if (e == cudaSuccess) e = bgw::band_sum_f64(sw, c->nb, nn, out + nn, c->st);         // every n''
    if (e == cudaSuccess) e = bgw::band_sum_f64(tv, c->nb, nn, out + 2 * nn, c->st);
    std::vector<double> h(3 * (size_t)nn);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "sigma_cohsex: kernels");
    const double scale = 1.0 / c->nk;
    for (int n = 0; n < nn; ++n) {
        sx[n] += -scale * h[n];
        coh[n] += 0.5 * scale * (h[nn + n] - h[2 * nn + n]);
    }
    return clean ? BGW_OK : BGW_W_ALIAS;
}

bgw_status bgw_bse_kernel(bgw_ctx c, int ik, int jk, const bgw_q *q0, const double *v0_coul, const bgw_q *qd,
                          const void *W_dev, int v0, int nv, int c0, int nc, void *KX_dev, void *KD_dev) {
    if (!c) return BGW_E_ARG;
    DeviceGuard dg(c->device);
    c->err.clear();
    if (c->prec != BGW_FP64) return c->fail(BGW_E_STATE, "bse_kernel: needs a BGW_FP64 context");
    if (ik < 0 || ik >= c->nk || jk < 0 || jk >= c->nk)
        return c->fail(BGW_E_ARG, "bse_kernel: k indices %d, %d out of range", ik, jk);
    if (nv < 1 || v0 < 0 || v0 + nv > c->nv || nc < 1 || c0 < 0 || c0 + nc > c->nc_max)
        return c->fail(BGW_E_ARG, "bse_kernel: band ranges outside the context's valence/conduction bands");
    if (KX_dev && (!q0 || !v0_coul)) return c->fail(BGW_E_ARG, "bse_kernel: K^X needs q0 and v(G)");
    if (KD_dev && (!qd || !W_dev)) return c->fail(BGW_E_ARG, "bse_kernel: K^D needs qd and W");
    const long P = (long)nv * nc;
    const double scale = 1.0 / c->nk;
    bool clean = true;
    cudaError_t e = cudaSuccess;
    if (KX_dev) {
        QState s;
        bgw_status st = prepare_q(c, q0, s, false);
        if (st != BGW_OK) return st;
        for (int g = 0; g < s.ng; ++g)
            if (!std::isfinite(v0_coul[g]) || v0_coul[g] < 0)
                return c->fail(BGW_E_ARG, "bse_kernel: v(G) must be finite and >= 0");
        int kp, G0[3];
        if (!find_umklapp(c, ik, s.q, kp, G0) || kp != ik || !find_umklapp(c, jk, s.q, kp, G0) || kp != jk)
            return c->fail(BGW_E_ARG, "bse_kernel: q0 must be a reciprocal lattice vector (k + q0 = k)");
        const size_t mb = 16 * (size_t)P * s.ng;
        e = c->nx_m1.ensure(mb, c->st);
        if (e == cudaSuccess) e = c->nx_m2.ensure(mb, c->st);
        if (e == cudaSuccess) e = c->nx_v.ensure(sizeof(double) * (size_t)s.ng, c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "bse_kernel: scratch");
        const int va = v0, ca = c->nv + c0;   // absolute band indices
        st = mtxel_into(c, "bse_kernel", s, ik, va, nv, ca, nc, c->nx_m1.p, clean);
        if (st == BGW_OK) st = mtxel_into(c, "bse_kernel", s, jk, va, nv, ca, nc, c->nx_m2.p, clean);
        if (st != BGW_OK) return st;
        e = cudaMemcpyAsync(c->nx_v.p, v0_coul, sizeof(double) * s.ng, cudaMemcpyHostToDevice, c->st);
        // KX[I][J] = (1/N_k) sum_G v(G) M_I(k_i, G) conj(M_J(k_j, G))
        if (e == cudaSuccess)
            e = bgw::zgemm_f64((int)P, (int)P, s.ng, c->nx_m1.p, s.ng, 1, false, c->nx_m2.p, 1, s.ng, true,
                               static_cast<const double *>(c->nx_v.p), KX_dev, P, 1, scale, 0.0, false, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);   // the host copy of v(G) has been read
        if (e != cudaSuccess) return c->cuda_fail(e, "bse_kernel: exchange");
    }
    if (KD_dev) {
        QState s;
        bgw_status st = prepare_q(c, qd, s, false);
        if (st != BGW_OK) return st;
        int kp, G0[3];
        if (!find_umklapp(c, ik, s.q, kp, G0) || kp != jk)
            return c->fail(BGW_E_ARG, "bse_kernel: k_i + qd must land on k_j");
        const size_t mcc = 16 * (size_t)nc * nc * s.ng, mvv = 16 * (size_t)nv * nv * s.ng;
        e = c->nx_m1.ensure(mcc, c->st);
        if (e == cudaSuccess) e = c->nx_m2.ensure(mvv, c->st);
        if (e == cudaSuccess) e = c->nx_y.ensure(mvv, c->st);
        if (e == cudaSuccess) e = c->nx_t.ensure(16 * (size_t)P * P, c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "bse_kernel: scratch");
        // M_cc'(k_i, qd, G) and M_vv'(k_i, qd, G): bands at k_i and at k_j
        st = mtxel_into(c, "bse_kernel", s, ik, c->nv + c0, nc, c->nv + c0, nc, c->nx_m1.p, clean);
        if (st == BGW_OK) st = mtxel_into(c, "bse_kernel", s, ik, v0, nv, v0, nv, c->nx_m2.p, clean);
        if (st != BGW_OK) return st;
        const int nv2 = nv * nv, nc2 = nc * nc;
        // Y[(v v')][G] = sum_G' W[G][G'] M_vv'(G')
        e = bgw::zgemm_f64(nv2, s.ng, s.ng, c->nx_m2.p, s.ng, 1, false, W_dev, 1, s.ng, false, nullptr, c->nx_y.p,
                           s.ng, 1, 1.0, 0.0, false, c->st);
        // T[(c c')][(v v')] = -(1/N_k) sum_G conj(M_cc'(G)) Y[(v v')][G]
        if (e == cudaSuccess)
            e = bgw::zgemm_f64(nc2, nv2, s.ng, c->nx_m1.p, s.ng, 1, true, c->nx_y.p, 1, s.ng, false, nullptr,
                               c->nx_t.p, nv2, 1, -scale, 0.0, false, c->st);
        if (e == cudaSuccess) e = bgw::bse_permute_f64(c->nx_t.p, nv, nc, KD_dev, c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "bse_kernel: direct");
    }
    return clean ? BGW_OK : BGW_W_ALIAS;
}

}  // extern "C"
