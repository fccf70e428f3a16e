// C ABI of libdfilt.so (declared in include/dfilt.h): argument checks on the host,
// workspace sizing, algorithm choice and kernel dispatch.  No entry point allocates
// or frees device memory.
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace dfilt;

// Device status word: first nonzero dfilt_status a kernel records wins.
__device__ int g_dfilt_status;

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int *g_status_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};
long long g_wait_limit = kDefaultWaitLimit;
int g_stall_drill = 0;
long long g_dbg_limit = 0;   // debug build: sample bound of the index checks (0: none)
bool g_numeric_check = false;

// NVTX range around an entry point (header-only NVTX: a no-op unless a profiler
// attaches)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Optional output check: records DFILT_ERR_NUMERIC in the status word when any of the
// n floats at p is not finite (grid-stride; vector loads where the pointer allows).
__global__ void check_finite_kernel(const float *__restrict__ p, int64_t n, int *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 4; i += stride) {
            const float4 v = __ldg(p4 + i);
            bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
        }
        for (int64_t i = n / 4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
            bad |= !isfinite(__ldg(p + i));
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
            bad |= !isfinite(__ldg(p + i));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(status, DFILT_ERR_NUMERIC);
}

cudaError_t check_finite(const float *p, int64_t n, int *status, int num_sms, cudaStream_t st) {
    if (!p || n <= 0) return cudaSuccess;
    const int64_t want = (n / 4 + 255) / 256;
    const int grid = (int)(want < 4LL * num_sms ? (want > 0 ? want : 1) : 4LL * num_sms);
    check_finite_kernel<<<grid, 256, 0, st>>>(p, n, status);
    note_launch();
    return cudaGetLastError();
}

struct DevInfo {
    int *status;
    int num_sms;
};

bool dev_info(DevInfo *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dfilt_status) != cudaSuccess) return false;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return false;
        g_status_addr[dev] = static_cast<int *>(p);
        g_num_sms[dev] = sms;
    }
    out->status = g_status_addr[dev];
    out->num_sms = g_num_sms[dev];
    return true;
}

struct Resolved {
    int algo;
    int precision;
    int fp64_opt;   // chunk-state scan option: -1 automatic per state bucket, 0 FP32, 1 FP64
    HiOpt hi;       // high-order path and scan span length
};

dfilt_status resolve(const dfilt_opts *o, int Mmax, Resolved *r) {
    dfilt_opts d;
    dfilt_default_opts(&d);
    if (!o) o = &d;
    if (o->algo < DFILT_ALGO_AUTO || o->algo > DFILT_ALGO_CHUNKED) return DFILT_ERR_INVALID_ARG;
    if (o->chunk_len != 0 && o->chunk_len != kL) return DFILT_ERR_UNSUPPORTED;
    if (o->fp64_scan < -1 || o->fp64_scan > 1) return DFILT_ERR_INVALID_ARG;
    if (o->path < DFILT_PATH_AUTO || o->path > DFILT_PATH_DECOUPLED) return DFILT_ERR_INVALID_ARG;
    if (o->span_tiles < 0 || o->span_tiles > 4096 || (o->span_tiles & (o->span_tiles - 1)) != 0)
        return DFILT_ERR_INVALID_ARG;
    r->hi.path = o->path;
    r->hi.span_tiles = o->span_tiles;
    r->algo = o->algo == DFILT_ALGO_AUTO ? DFILT_ALGO_CHUNKED : o->algo;
    r->precision = o->precision;
    if (r->algo == DFILT_ALGO_CHUNKED) {
        if (o->precision != DFILT_PREC_TF32 && o->precision != DFILT_PREC_TF32X3)
            return DFILT_ERR_UNSUPPORTED;
    } else if (o->precision != DFILT_PREC_FP32 && o->precision != DFILT_PREC_TF32 &&
               o->precision != DFILT_PREC_TF32X3) {
        return DFILT_ERR_INVALID_ARG;
    }
    r->fp64_opt = o->fp64_scan;
    return DFILT_OK;
}

dfilt_status check_orders(int N, int M) {
    if (M > 64) return DFILT_ERR_UNSUPPORTED;
    if (M < 1 || N < 0 || N > M) return DFILT_ERR_INVALID_ARG;
    return DFILT_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

dfilt_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DFILT_OK;
    if (e == cudaErrorNotSupported) return DFILT_ERR_UNSUPPORTED;
    return DFILT_ERR_CUDA;
}

void sizes(const Resolved &r, int64_t B, int64_t total, int Mmax, bool ragged, size_t *fwd,
           size_t *saved, size_t *bwd) {
    size_t f = 0, s = 0, w = 0;
    if (r.algo == DFILT_ALGO_CHUNKED) {
        f = chunk_fwd_ws_bytes(B, total, Mmax, r.fp64_opt, ragged, r.hi);
        s = chunk_saved_bytes(B, total, Mmax, r.fp64_opt, ragged, r.hi);
        w = chunk_bwd_ws_bytes(B, total, Mmax, r.fp64_opt, ragged, r.hi);
    }
    if (fwd) *fwd = f;
    if (saved) *saved = s;
    if (bwd) *bwd = w;
}

Batch make_batch(const DevInfo &di, const int64_t *offsets, const int *Ms, const int *Ns,
                 int64_t B, int64_t T, int64_t total, int N, int M, int Nmax, int Mmax) {
    Batch bt;
    bt.offsets = offsets;
    bt.Ms = Ms;
    bt.Ns = Ns;
    bt.B = B;
    bt.T = T;
    bt.total = total;
    bt.M = M;
    bt.N = N;
    bt.Mstride = Mmax;
    bt.Nstride = Nmax + 1;
    bt.status = di.status;
    bt.list = nullptr;
    bt.list_range = nullptr;
    bt.fwd_stride = 0;
    bt.bwd_stride = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        bt.wait_limit = g_wait_limit;
        bt.stall_drill = g_stall_drill;
        bt.dbg_limit = g_dbg_limit > 0 && g_dbg_limit < total ? g_dbg_limit : total;
    }
    return bt;
}

dfilt_status do_forward(const float *x, const float *b, const float *a, const float *zi, float *y,
                        void *saved, void *ws, size_t ws_bytes, const Batch &bt, int Mmax,
                        const Resolved &r, const DevInfo &di, cudaStream_t st) {
    if (bt.B == 0 || bt.total == 0) return DFILT_OK;
    if (r.algo == DFILT_ALGO_SEQUENTIAL) {
        timing_mark(0, 0, st);
        const cudaError_t e = launch_seq_fwd(x, b, a, zi, y, bt, Mmax, st);
        timing_mark(0, 1, st);
        return cuda_status(e);
    }
    const bool ragged = bt.offsets != nullptr;
    size_t need = chunk_fwd_ws_bytes(bt.B, bt.total, Mmax, r.fp64_opt, ragged, r.hi);
    if (ws_bytes < need || (need && !ws)) return DFILT_ERR_WORKSPACE;
    if (!aligned16(ws) || (saved && !aligned16(saved))) return DFILT_ERR_INVALID_ARG;
    return cuda_status(launch_chunk_fwd(x, b, a, zi, y, static_cast<float *>(saved), ws, bt, Mmax,
                                        r.fp64_opt, r.precision, di.num_sms, st, r.hi));
}

bool numeric_check_on() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_numeric_check;
}

// the optional finite-output check after a successful enqueue
dfilt_status checked(dfilt_status s, const float *const *outs, const int64_t *sizes, int nout,
                     const DevInfo &di, cudaStream_t st) {
    if (s != DFILT_OK || !numeric_check_on()) return s;
    for (int k = 0; k < nout; ++k) {
        const cudaError_t e = check_finite(outs[k], sizes[k], di.status, di.num_sms, st);
        if (e != cudaSuccess) return DFILT_ERR_CUDA;
    }
    return DFILT_OK;
}

dfilt_status do_backward(const float *gy, const float *x, const float *y, const float *b,
                         const float *a, const void *saved, float *gx, float *gb, float *ga,
                         float *gzi, void *ws, size_t ws_bytes, const Batch &bt, int Mmax,
                         const Resolved &r, const DevInfo &di, cudaStream_t st) {
    if (bt.B == 0) return DFILT_OK;
    if (r.algo == DFILT_ALGO_SEQUENTIAL) {
        if (!y) return DFILT_ERR_INVALID_ARG;
        timing_mark(1, 0, st);
        const cudaError_t e = launch_seq_bwd(gy, x, y, b, a, gx, gb, ga, gzi, bt, Mmax, st);
        timing_mark(1, 1, st);
        return cuda_status(e);
    }
    if (!y && !saved) return DFILT_ERR_INVALID_ARG;
    const bool ragged = bt.offsets != nullptr;
    size_t need = chunk_bwd_ws_bytes(bt.B, bt.total, Mmax, r.fp64_opt, ragged, r.hi);
    if (ws_bytes < need || (need && !ws)) return DFILT_ERR_WORKSPACE;
    if (!aligned16(ws) || (saved && !aligned16(saved))) return DFILT_ERR_INVALID_ARG;
    return cuda_status(launch_chunk_bwd(gy, x, y, b, a, static_cast<const float *>(saved), gx, gb,
                                        ga, gzi, ws, bt, Mmax, r.fp64_opt, r.precision,
                                        di.num_sms, st, r.hi));
}

// ---- kernel timing: event pairs around each call's main kernel --------------------
constexpr int kTimingSlots = 4096;
struct TimingSlot {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = -1;
    int dir = 0;
    int state = 0;   // 0 free, 1 started, 2 complete
};
std::mutex g_tmu;
bool g_timing_on = false;
TimingSlot g_slots[kTimingSlots];
constexpr int kTimingClasses = 8;
thread_local int t_pending[kTimingClasses] = {-1, -1, -1, -1, -1, -1, -1, -1};
std::atomic<long long> g_launches{0};

}  // namespace

namespace dfilt {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void timing_mark(int dir, int phase, cudaStream_t st) {
    if (dir < 0 || dir >= kTimingClasses) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    if (!g_timing_on) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (phase == 0) {
        t_pending[dir] = -1;
        for (int i = 0; i < kTimingSlots; ++i) {
            TimingSlot &sl = g_slots[i];
            if (sl.state != 0) continue;
            if (sl.dev != dev) {
                if (sl.e0) cudaEventDestroy(sl.e0);
                if (sl.e1) cudaEventDestroy(sl.e1);
                sl.e0 = sl.e1 = nullptr;
                if (cudaEventCreate(&sl.e0) != cudaSuccess || cudaEventCreate(&sl.e1) != cudaSuccess)
                    return;
                sl.dev = dev;
            }
            if (cudaEventRecord(sl.e0, st) != cudaSuccess) return;
            sl.dir = dir;
            sl.state = 1;
            t_pending[dir] = i;
            return;
        }
    } else {
        const int i = t_pending[dir];
        t_pending[dir] = -1;
        if (i < 0 || g_slots[i].state != 1) return;
        if (cudaEventRecord(g_slots[i].e1, st) != cudaSuccess) {
            g_slots[i].state = 0;
            return;
        }
        g_slots[i].state = 2;
    }
}
}  // namespace dfilt

namespace dfilt {
// Status word, SM count and wait settings of the current device, for entry points
// defined in other translation units.
bool api_launch_context(int **status, int *num_sms, long long *wait_limit, int *stall_drill) {
    DevInfo di;
    if (!dev_info(&di)) return false;
    *status = di.status;
    *num_sms = di.num_sms;
    std::lock_guard<std::mutex> lk(g_mu);
    *wait_limit = g_wait_limit;
    *stall_drill = g_stall_drill;
    return true;
}

// The finite-output check for an entry point defined outside this file (one output).
dfilt_status api_check_output(const float *out, int64_t n, cudaStream_t st) {
    if (!numeric_check_on()) return DFILT_OK;
    DevInfo di;
    if (!dev_info(&di)) return DFILT_ERR_CUDA;
    const float *outs[1] = {out};
    const int64_t sizes[1] = {n};
    return checked(DFILT_OK, outs, sizes, 1, di, st);
}
}  // namespace dfilt

extern "C" {

int dfilt_version(void) { return 100; }

const char *dfilt_status_string(dfilt_status s) {
    switch (s) {
        case DFILT_OK: return "DFILT_OK";
        case DFILT_ERR_INVALID_ARG: return "DFILT_ERR_INVALID_ARG";
        case DFILT_ERR_UNSUPPORTED: return "DFILT_ERR_UNSUPPORTED";
        case DFILT_ERR_CUDA: return "DFILT_ERR_CUDA";
        case DFILT_ERR_TIMEOUT: return "DFILT_ERR_TIMEOUT";
        case DFILT_ERR_NUMERIC: return "DFILT_ERR_NUMERIC";
        case DFILT_ERR_WORKSPACE: return "DFILT_ERR_WORKSPACE";
        case DFILT_ERR_BOUNDS: return "DFILT_ERR_BOUNDS";
    }
    return "DFILT_ERR_UNKNOWN";
}

dfilt_status dfilt_default_opts(dfilt_opts *o) {
    if (!o) return DFILT_ERR_INVALID_ARG;
    o->algo = DFILT_ALGO_AUTO;
    o->precision = DFILT_PREC_TF32X3;
    o->chunk_len = 0;
    o->fp64_scan = -1;
    o->path = DFILT_PATH_AUTO;
    o->span_tiles = 0;
    return DFILT_OK;
}

dfilt_status dfilt_workspace_size(int64_t B, int64_t T, int N, int M, const dfilt_opts *opts,
                                  size_t *fwd_ws, size_t *saved, size_t *bwd_ws) {
    if (B < 0 || T < 0) return DFILT_ERR_INVALID_ARG;
    dfilt_status s = check_orders(N, M);
    if (s) return s;
    Resolved r;
    if ((s = resolve(opts, M, &r))) return s;
    sizes(r, B, B * T, M, false, fwd_ws, saved, bwd_ws);
    return DFILT_OK;
}

dfilt_status dfilt_workspace_size_ragged(int64_t B, int64_t total, int Nmax, int Mmax,
                                         const dfilt_opts *opts, size_t *fwd_ws, size_t *saved,
                                         size_t *bwd_ws) {
    if (B < 0 || total < 0) return DFILT_ERR_INVALID_ARG;
    dfilt_status s = check_orders(Nmax, Mmax);
    if (s) return s;
    Resolved r;
    if ((s = resolve(opts, Mmax, &r))) return s;
    sizes(r, B, total, Mmax, true, fwd_ws, saved, bwd_ws);
    return DFILT_OK;
}

dfilt_status dfilt_forward(const float *x, const float *b, const float *a, const float *zi,
                           float *y, void *saved, void *ws, size_t ws_bytes, int64_t B, int64_t T,
                           int N, int M, const dfilt_opts *opts, void *stream) {
    NvtxRange nv("dfilt_forward");
    if (B < 0 || T < 0) return DFILT_ERR_INVALID_ARG;
    dfilt_status s = check_orders(N, M);
    if (s) return s;
    if (B > 0 && T > 0 && (!x || !b || !a || !y)) return DFILT_ERR_INVALID_ARG;
    Resolved r;
    if ((s = resolve(opts, M, &r))) return s;
    DevInfo di;
    if (!dev_info(&di)) return DFILT_ERR_CUDA;
    Batch bt = make_batch(di, nullptr, nullptr, nullptr, B, T, B * T, N, M, N, M);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *outs[1] = {y};
    const int64_t n[1] = {B * T};
    return checked(do_forward(x, b, a, zi, y, saved, ws, ws_bytes, bt, M, r, di, st), outs, n, 1,
                   di, st);
}

dfilt_status dfilt_backward(const float *gy, const float *x, const float *y, const float *b,
                            const float *a, const float *zi, const void *saved, float *gx,
                            float *gb, float *ga, float *gzi, void *ws, size_t ws_bytes, int64_t B,
                            int64_t T, int N, int M, const dfilt_opts *opts, void *stream) {
    NvtxRange nv("dfilt_backward");
    (void)zi;   // carried inside `saved` (chunk 0's entry state) when y is recomputed
    if (B < 0 || T < 0) return DFILT_ERR_INVALID_ARG;
    dfilt_status s = check_orders(N, M);
    if (s) return s;
    if (B > 0 && (!gy || !x || !b || !a)) return DFILT_ERR_INVALID_ARG;
    Resolved r;
    if ((s = resolve(opts, M, &r))) return s;
    DevInfo di;
    if (!dev_info(&di)) return DFILT_ERR_CUDA;
    Batch bt = make_batch(di, nullptr, nullptr, nullptr, B, T, B * T, N, M, N, M);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *outs[4] = {gx, gb, ga, gzi};
    const int64_t n[4] = {B * T, B * (N + 1), B * M, B * M};
    return checked(do_backward(gy, x, y, b, a, saved, gx, gb, ga, gzi, ws, ws_bytes, bt, M, r, di, st),
                   outs, n, 4, di, st);
}

dfilt_status dfilt_forward_ragged(const float *x, const int64_t *offsets, const int *Ms,
                                  const int *Ns, const float *b, const float *a, const float *zi,
                                  float *y, void *saved, void *ws, size_t ws_bytes, int64_t B,
                                  int64_t total, int Nmax, int Mmax, const dfilt_opts *opts,
                                  void *stream) {
    NvtxRange nv("dfilt_forward_ragged");
    if (B < 0 || total < 0) return DFILT_ERR_INVALID_ARG;
    dfilt_status s = check_orders(Nmax, Mmax);
    if (s) return s;
    if (B > 0 && (!offsets || !Ms || !Ns || !b || !a || (total > 0 && (!x || !y))))
        return DFILT_ERR_INVALID_ARG;
    Resolved r;
    if ((s = resolve(opts, Mmax, &r))) return s;
    DevInfo di;
    if (!dev_info(&di)) return DFILT_ERR_CUDA;
    Batch bt = make_batch(di, offsets, Ms, Ns, B, 0, total, Nmax, Mmax, Nmax, Mmax);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *outs[1] = {y};
    const int64_t n[1] = {total};
    return checked(do_forward(x, b, a, zi, y, saved, ws, ws_bytes, bt, Mmax, r, di, st), outs, n,
                   1, di, st);
}

dfilt_status dfilt_backward_ragged(const float *gy, const float *x, const float *y,
                                   const int64_t *offsets, const int *Ms, const int *Ns,
                                   const float *b, const float *a, const float *zi,
                                   const void *saved, float *gx, float *gb, float *ga, float *gzi,
                                   void *ws, size_t ws_bytes, int64_t B, int64_t total, int Nmax,
                                   int Mmax, const dfilt_opts *opts, void *stream) {
    NvtxRange nv("dfilt_backward_ragged");
    (void)zi;
    if (B < 0 || total < 0) return DFILT_ERR_INVALID_ARG;
    dfilt_status s = check_orders(Nmax, Mmax);
    if (s) return s;
    if (B > 0 && (!offsets || !Ms || !Ns || !b || !a || (total > 0 && (!gy || !x))))
        return DFILT_ERR_INVALID_ARG;
    Resolved r;
    if ((s = resolve(opts, Mmax, &r))) return s;
    DevInfo di;
    if (!dev_info(&di)) return DFILT_ERR_CUDA;
    Batch bt = make_batch(di, offsets, Ms, Ns, B, 0, total, Nmax, Mmax, Nmax, Mmax);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *outs[4] = {gx, gb, ga, gzi};
    const int64_t n[4] = {total, B * (Nmax + 1), B * Mmax, B * Mmax};
    return checked(do_backward(gy, x, y, b, a, saved, gx, gb, ga, gzi, ws, ws_bytes, bt, Mmax, r,
                               di, st),
                   outs, n, 4, di, st);
}

dfilt_status dfilt_sync_status(void *stream) {
    DevInfo di;
    if (!dev_info(&di)) return DFILT_ERR_CUDA;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return DFILT_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, di.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return DFILT_ERR_CUDA;
    if (v != 0 && cudaMemset(di.status, 0, sizeof(int)) != cudaSuccess) return DFILT_ERR_CUDA;
    return static_cast<dfilt_status>(v);
}

dfilt_status dfilt_kernel_timing(int enable) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing_on = enable != 0;
    for (TimingSlot &sl : g_slots)
        if (sl.state != 0) sl.state = 0;
    return DFILT_OK;
}

// sums of the recorded pairs per class (then discarded)
static dfilt_status timing_collect(double *ms, int *n) {
    std::lock_guard<std::mutex> lk(g_tmu);
    dfilt_status st = DFILT_OK;
    for (int k = 0; k < kTimingClasses; ++k) {
        ms[k] = 0.0;
        n[k] = 0;
    }
    for (TimingSlot &sl : g_slots) {
        if (sl.state != 2) {
            sl.state = 0;
            continue;
        }
        float t = 0.f;
        if (cudaEventSynchronize(sl.e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, sl.e0, sl.e1) != cudaSuccess) {
            st = DFILT_ERR_CUDA;
        } else {
            ms[sl.dir] += t;
            ++n[sl.dir];
        }
        sl.state = 0;
    }
    return st;
}

dfilt_status dfilt_kernel_timing_read(double *fwd_ms, int *fwd_calls, double *bwd_ms,
                                      int *bwd_calls) {
    double ms[kTimingClasses];
    int n[kTimingClasses];
    const dfilt_status st = timing_collect(ms, n);
    if (fwd_ms) *fwd_ms = ms[0];
    if (fwd_calls) *fwd_calls = n[0];
    if (bwd_ms) *bwd_ms = ms[1];
    if (bwd_calls) *bwd_calls = n[1];
    return st;
}

dfilt_status dfilt_kernel_timing_read_classes(double *ms, int *calls) {
    if (!ms || !calls) return DFILT_ERR_INVALID_ARG;
    return timing_collect(ms, calls);
}

dfilt_status dfilt_tuning_set(int state_bucket, int span_tiles, int chains_per_sm) {
    return dfilt::hi_tuning_set(state_bucket, span_tiles, chains_per_sm) ? DFILT_OK
                                                                         : DFILT_ERR_INVALID_ARG;
}

dfilt_status dfilt_tuning_get(int state_bucket, int *span_tiles, int *chains_per_sm) {
    if (chunk_bucket(state_bucket) != state_bucket) return DFILT_ERR_INVALID_ARG;
    dfilt::hi_tuning_get(state_bucket, span_tiles, chains_per_sm);
    return DFILT_OK;
}

dfilt_status dfilt_launch_count(int64_t *n) {
    if (!n) return DFILT_ERR_INVALID_ARG;
    *n = (int64_t)g_launches.load(std::memory_order_relaxed);
    return DFILT_OK;
}

dfilt_status dfilt_set_numeric_check(int enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_numeric_check = enable != 0;
    return DFILT_OK;
}

int dfilt_debug_build(void) {
#ifdef DFILT_DEBUG
    return 1;
#else
    return 0;
#endif
}

dfilt_status dfilt_debug_set_limit(int64_t samples) {
#ifdef DFILT_DEBUG
    std::lock_guard<std::mutex> lk(g_mu);
    g_dbg_limit = samples > 0 ? (long long)samples : 0;
    return DFILT_OK;
#else
    (void)samples;
    return DFILT_ERR_UNSUPPORTED;
#endif
}

dfilt_status dfilt_set_wait_limit(int64_t iters) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_stall_drill = iters < 0 ? 1 : 0;
    g_wait_limit = iters == 0 ? kDefaultWaitLimit : (long long)(iters < 0 ? -iters : iters);
    return DFILT_OK;
}

}  // extern "C"
