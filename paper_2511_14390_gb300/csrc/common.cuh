// Device helpers shared by the dfilt kernels: status word, bounded waits, and
// thin inline-PTX wrappers for sm_103a (mbarrier, cp.async, tcgen05, proxy fences).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/dfilt.h"

namespace dfilt {

// ---------------------------------------------------------------------------
// Device status word (first nonzero code wins; lives in the API translation unit,
// its address reaches every kernel through Batch::status) and the default cap on
// bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

constexpr long long kDefaultWaitLimit = 1ll << 26;   // polls; ~seconds at worst

// ---------------------------------------------------------------------------
// Host-side launch arguments.  One struct serves fixed-shape and ragged batches:
// offsets == nullptr means channel i owns [i*T, (i+1)*T) and every channel has
// orders (M, N).
// ---------------------------------------------------------------------------
struct Batch {
    const int64_t *offsets;   // [B+1] or nullptr
    const int *Ms;            // [B] or nullptr
    const int *Ns;            // [B] or nullptr
    int64_t B;
    int64_t T;                // fixed shape only
    int64_t total;            // samples in the packed signal
    int M, N;                 // fixed-shape orders
    int Mstride, Nstride;     // row strides of a/zi and b (Mmax, Nmax+1)
    int *status;              // device status word
    long long wait_limit;     // cap on polls of any bounded wait
    int stall_drill;          // test mode: also wait on a barrier nothing signals
    int64_t dbg_limit;        // debug build: samples the index checks allow (<= total)
    // Optional sub-list of channels for one launch (a state-order bucket of a ragged
    // batch): work item c is channel list[list_range[0] + c], c < list_range[1] -
    // list_range[0].  nullptr: work item c is channel c < B.
    const int *list;
    const int *list_range;
    // Byte strides of the per-channel table records (0: the launch's own record size;
    // set when buckets of different sizes share one workspace).
    int64_t fwd_stride, bwd_stride;
};

struct Channel {
    int64_t off;
    int64_t len;
    int M, N;
};

// Channel of work item c of a launch; false once the launch's work is exhausted.
__device__ __forceinline__ bool work_channel(const Batch &bt, int64_t c, int64_t *ch) {
    if (!bt.list) {
        *ch = c;
        return c < bt.B;
    }
    const int lo = bt.list_range[0], hi = bt.list_range[1];
    if (c >= (int64_t)(hi - lo)) return false;
    *ch = bt.list[lo + c];
    return true;
}

__device__ __forceinline__ Channel channel_of(const Batch &bt, int64_t i) {
    Channel c;
    if (bt.offsets) {
        int64_t o0 = bt.offsets[i], o1 = bt.offsets[i + 1];
        // Clamp so a malformed offsets array can never address outside [0, total).
        bool bad = (o0 < 0) | (o1 < o0) | (o1 > bt.total);
        if (bad) set_status(bt.status, DFILT_ERR_INVALID_ARG);
        o0 = o0 < 0 ? 0 : (o0 > bt.total ? bt.total : o0);
        o1 = o1 < o0 ? o0 : (o1 > bt.total ? bt.total : o1);
        c.off = o0;
        c.len = o1 - o0;
        int m = bt.Ms[i], n = bt.Ns[i];
        if (m < 1 || m > bt.Mstride || n < 0 || n > m) {
            set_status(bt.status, DFILT_ERR_INVALID_ARG);
            m = m < 1 ? 1 : (m > bt.Mstride ? bt.Mstride : m);
            n = n < 0 ? 0 : (n > m ? m : n);
        }
        c.M = m;
        c.N = n;
    } else {
        c.off = i * bt.T;
        c.len = bt.T;
        c.M = bt.M;
        c.N = bt.N;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Shared-memory address helpers and async copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// The dynamic shared-memory array advanced to the next 1024-byte boundary (the repeat of
// the 128-byte swizzle).  The step is added to the array's own address rather than
// formed by rounding an integer, so the result still derives from a shared-memory array
// and the compiler emits shared-memory loads and stores for every access through it
// (a pointer rebuilt from an integer is generic: each access then goes through the
// generic path, with its longer latency, on the long scoreboard).
__device__ __forceinline__ char *smem_align1024(char *raw) {
    const uint32_t s = smem_u32(raw);
    return raw + (((s + 1023u) & ~1023u) - s);
}

// 16-byte async global->shared copy; bytes beyond src_bytes (0..16) are zero-filled.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
// 4-byte async copy (for signals whose channel start is not 16-byte aligned).
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// all but this thread's most recent cp.async group have landed
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// Arrive on `bar` once this thread's earlier cp.async copies have landed (the arrival is
// counted in the barrier's initial count).
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the async proxy
// (tensor-core operand reads).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// Non-blocking probe of an mbarrier phase (so that a poll cap is a real bound).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase: at most `limit` polls.  Returns false when the
// phase did not complete in time (the caller records DFILT_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// Arrive and announce `bytes` of transaction (TMA) data the current phase must receive.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// ---------------------------------------------------------------------------
// TMA (tensor bulk copies) and bulk-group completion
// ---------------------------------------------------------------------------
// 3-D tiled load global -> shared, completion counted on an mbarrier (bytes).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
// Untiled bulk copy global -> shared (both addresses 16-byte aligned, size a multiple
// of 16), completion counted on an mbarrier (bytes).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// 3-D tiled store shared -> global (bulk async-group completion).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int c0, int c1, int c2,
                                             uint32_t src) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(c0), "r"(c1), "r"(c2), "r"(src)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// all committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read0() {
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// all but the most recent committed bulk store group have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read1() {
    asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
}
// all committed bulk stores are complete
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// tcgen05 (5th-generation tensor cores, accumulators in tensor memory)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, TF32 operands, FP32 accumulate.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem]^T, TF32 operands, FP32 accumulate; A's row r is TMEM
// lane r, its K elements consecutive 32-bit columns from a_tmem.
__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                                uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive once on `bar` when every tcgen05 operation this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_tf32_m128(int n) {
    return (1u << 4)                         // D format F32
           | (2u << 7)                       // A format TF32
           | (2u << 10)                      // B format TF32
           | ((uint32_t)(n >> 3) << 17)      // N / 8
           | ((uint32_t)(128 >> 4) << 24);   // M / 16
}

// Shared-memory matrix descriptor, K-major with the 128-byte swizzle: rows of 128 B
// (32 fp32), 8-row atoms of 1024 B (stride-dimension offset), base 1024-B aligned.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;               // leading-dimension offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride-dimension offset: 1024 B per 8 rows
    d |= (uint64_t)1 << 46;               // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}

// Byte offset of element (row r, k in [0,32)) inside one 128-B-swizzled K block.
__host__ __device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) << 4)) + ((k & 3) << 2));
}

// 32 lanes x 16 consecutive 32-bit columns from tensor memory.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
// 32 lanes x 16 consecutive 32-bit columns into tensor memory.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// fp32 -> (hi, lo) with hi exactly representable in TF32 (low 13 mantissa bits cleared)
// and lo = x - hi (exact in fp32); the tensor core sees hi exactly and lo to TF32.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

}  // namespace dfilt
