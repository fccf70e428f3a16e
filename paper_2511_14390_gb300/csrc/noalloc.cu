// dfilt_forward_noalloc: the chunked forward with its scratch in a fixed, statically
// allocated device array instead of a caller-provided workspace.
//
// Who needs it: callers that must not allocate device memory while they run, such as
// a real-time audio callback (cudaMalloc/cudaFree may synchronise the device and have
// unbounded latency) or a host program that has no device allocator of its own to
// obtain a workspace from.  They pass only inputs and outputs.
//
// The scratch holds the per-channel coefficient tables and the channel work counter
// of the chunked forward (exactly what dfilt_forward keeps in `ws`).  It lives in
// g_noalloc_scratch below: kNoallocScratchBytes (4 MiB) per GPU that loads this
// library, held until the process exits.  The first call on a device looks up the
// array's device address with cudaGetSymbolAddress (with that device current) and
// caches it; make that first call before any stream capture.  Every call reuses the
// same array, so calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.  Nothing
// in it needs clearing by the host: the setup kernel rewrites the tables and resets
// the work counter at the start of every call.
#include <mutex>

#include "chunk.cuh"

namespace dfilt {
// Launch context shared with the other entry points (defined in api.cu).
bool api_launch_context(int **status, int *num_sms, long long *wait_limit, int *stall_drill);
// The optional finite-output check of the other entry points (a no-op while it is off).
dfilt_status api_check_output(const float *out, int64_t n, cudaStream_t st);
}  // namespace dfilt

using namespace dfilt;

namespace {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDev] = {};

// Device address of the scratch array for the current device (once per device).
void *noalloc_scratch() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
        g_noalloc_addr[dev] = p;
    }
    return g_noalloc_addr[dev];
}

}  // namespace

extern "C" dfilt_status dfilt_forward_noalloc(const float *x, const float *b, const float *a,
                                              const float *zi, float *y, int64_t B, int64_t T,
                                              int N, int M, const dfilt_opts *opts,
                                              void *stream) {
    if (B < 0 || T < 0) return DFILT_ERR_INVALID_ARG;
    if (M > 64) return DFILT_ERR_UNSUPPORTED;
    if (M < 1 || N < 0 || N > M) return DFILT_ERR_INVALID_ARG;
    if (B > 0 && T > 0 && (!x || !b || !a || !y)) return DFILT_ERR_INVALID_ARG;
    dfilt_opts o;
    dfilt_default_opts(&o);
    if (opts) o = *opts;
    if (o.algo != DFILT_ALGO_AUTO && o.algo != DFILT_ALGO_CHUNKED) return DFILT_ERR_INVALID_ARG;
    if (o.chunk_len != 0 && o.chunk_len != kL) return DFILT_ERR_UNSUPPORTED;
    if (o.fp64_scan < -1 || o.fp64_scan > 1) return DFILT_ERR_INVALID_ARG;
    if (o.precision != DFILT_PREC_TF32 && o.precision != DFILT_PREC_TF32X3)
        return DFILT_ERR_UNSUPPORTED;
    // Capacity check before touching the device: the tables for B channels must fit.
    // (the single-kernel chunked path: its scratch is the per-channel tables alone)
    HiOpt ho;
    ho.path = DFILT_PATH_FUSED;
    if (chunk_fwd_ws_bytes(B, B * T, M, o.fp64_scan, false, ho) > kNoallocScratchBytes)
        return DFILT_ERR_WORKSPACE;
    if (B == 0 || T == 0) return DFILT_OK;
    int *status = nullptr, num_sms = 0, drill = 0;
    long long wait_limit = 0;
    if (!api_launch_context(&status, &num_sms, &wait_limit, &drill)) return DFILT_ERR_CUDA;
    void *scratch = noalloc_scratch();
    if (!scratch) return DFILT_ERR_CUDA;
    Batch bt;
    bt.offsets = nullptr;
    bt.Ms = nullptr;
    bt.Ns = nullptr;
    bt.B = B;
    bt.T = T;
    bt.total = B * T;
    bt.M = M;
    bt.N = N;
    bt.Mstride = M;
    bt.Nstride = N + 1;
    bt.status = status;
    bt.wait_limit = wait_limit;
    bt.stall_drill = drill;
    bt.dbg_limit = B * T;
    bt.list = nullptr;
    bt.list_range = nullptr;
    bt.fwd_stride = 0;
    bt.bwd_stride = 0;
    const cudaError_t e = launch_chunk_fwd(x, b, a, zi, y, nullptr, scratch, bt, M, o.fp64_scan,
                                           o.precision, num_sms, static_cast<cudaStream_t>(stream), ho);
    if (e == cudaSuccess) return api_check_output(y, B * T, static_cast<cudaStream_t>(stream));
    return e == cudaErrorNotSupported ? DFILT_ERR_UNSUPPORTED : DFILT_ERR_CUDA;
}
