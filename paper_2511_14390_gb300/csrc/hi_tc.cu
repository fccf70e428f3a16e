// Decoupled high-order path, tensor-core tile passes (sm_103a).  Every tile (128 chunks
// x 64 samples of one channel) is independent here, since the chunk states come from
// the scan kernel: a persistent CTA takes tiles from a counter, in channel order, and
// rebuilds its B operand only when the channel changes.
//
//   Y pass             D = X T_g^T           N = 64   -> y = D + O_L S_c
//   U pass             D = G [T_g^a ; T_h^a]^T  N = 128 -> grad_x = D[:, 0:64) +
//                      O^gx S'_c and u = D[:, 64:128) + O^u S'_c; then the lag sums of
//                      grad_b, grad_a from u (kept in tensor memory with its tail
//                      u[64..64+MB) = S'_c); one partial per tile (fixed order)
// The free responses O_L S_c, O^u S'_c and O^gx S'_c are added on the CUDA cores in FP32,
// per chunk row: the chunk states of high-order filters are large numbers whose
// combination cancels, and the split-TF32 product (about 21 bits per operand) would cost
// digits there that FP32 FMAs keep.  For the same reason grad_x comes from the impulse
// response of B/A directly, not as B applied to the all-pole adjoint u (which can be far
// larger than grad_x when zeros of B sit near poles of A).
//
// Operands: K-major, 128-byte swizzle, TF32 split in three products (hi*hi + hi*lo +
// lo*hi) or one; the raw FP32 words serve as the A hi part (the tensor cores read a
// TF32 operand's upper 19 bits, which is the hi part of the split).
#include <cstring>

#include "hi.cuh"

#ifndef DFILT_MB
#error "compile once per state bucket with -DDFILT_MB=<8|16|32|64>"
#endif

namespace dfilt {

namespace {

using hi::Plan;
// threads per CTA: one per chunk row, two in the U pass (each takes half of a row's
// columns and lag products, so that eight warps hide the latencies of its longer epilogue)
template <int MODE>
__host__ __device__ constexpr int threads_of() { return MODE == hi::kU ? 256 : 128; }
constexpr uint32_t kKBlock = kChunks * 128;   // one 32-wide K block of the A operand

template <int MB, int MODE>
struct TcSmem {
    using Tab = ChunkTab<MB>;
    static_assert(MODE == hi::kY || MODE == hi::kU, "tile passes: Y and U");
    static constexpr bool OUT = true;                             // y or u rows
    static constexpr int N = MODE == hi::kU ? 2 * kL : kL;        // MMA N
    static constexpr int KTOT = kL;
    static constexpr int KB = 2;                                  // K blocks of 32
    static constexpr uint32_t BBLK = (uint32_t)N * 128;           // bytes of one B K block
    static constexpr uint32_t BHI = 0;
    static constexpr uint32_t BLO = KB * BBLK;
    // free-response tables [L][MB] f32: O_L (Y pass), or O^u then O^gx (U pass)
    static constexpr int NOT = MODE == hi::kU ? 2 : (OUT ? 1 : 0);
    static constexpr uint32_t OT = 2 * KB * BBLK;
    static constexpr uint32_t A0 = (OT + NOT * kL * MB * 4 + 1023) / 1024 * 1024;
    static constexpr uint32_t AHI = A0;
    static constexpr uint32_t ALO = A0 + KB * kKBlock;
    static constexpr uint32_t AEND = A0 + 2 * KB * kKBlock;
    // U pass: the x and y tiles (256-byte rows), loaded with the gy tile into their own
    // buffers where shared memory allows, else over the A operand once it is consumed
    static constexpr int KBLK = (MB + 1 + 15) / 16;               // lag blocks of 16
    static constexpr uint32_t XY_BYTES = 2u * kChunks * kL * 4;
    static constexpr uint32_t RED_BYTES = MODE == hi::kU ? 8u * KBLK * 32 * 4 : 0u;   // 8 warps
    static constexpr bool SEPXY =
        MODE == hi::kU && AEND + XY_BYTES + RED_BYTES + 32 + 1024 <= pipe::kSmemMax;
    static constexpr uint32_t XT = SEPXY ? AEND : A0;
    static constexpr uint32_t YT = XT + (uint32_t)kChunks * kL * 4;
    static constexpr uint32_t RED = SEPXY ? AEND + XY_BYTES : AEND;
    static constexpr uint32_t MISC = RED + RED_BYTES;
    // misc: mbarrier (8) | drill mbarrier (8) | tmem base (4) | ok flag (4) | work item (8)
    static constexpr uint32_t BYTES = MISC + 32;
    static constexpr uint32_t ALLOC = BYTES + 1024;
    // U pass tensor memory: grad_x [0, 64), then the adjoint window u_ext from column 64:
    // u[0..64), S'[0..MB), zeros (the lag windows read columns below
    // 64 + 16 (KBLK + 2) + 32)
    static constexpr int UEND = kL + 16 * (KBLK + 2) + 32;
    static constexpr uint32_t TMEM_COLS = MODE == hi::kU ? 256 : (N < 32 ? 32 : N);
    static_assert(MODE != hi::kU || UEND <= 256, "tensor-memory window");
};

// byte offset of 16-byte piece j of row r in a 256-byte-row staging tile
__device__ __forceinline__ uint32_t rowp(int r, int j) { return (uint32_t)(r * 256 + ((j ^ (r & 15)) << 4)); }

template <int MB, int MODE>
__global__ void __launch_bounds__(threads_of<MODE>(), 1)
    hi_tc_kernel(HiArgs h, Batch bt, int sig_al, int out_al, int xy_al, int st_al) {
    using Tab = ChunkTab<MB>;
    using SM = TcSmem<MB, MODE>;
    constexpr int kThreads = threads_of<MODE>();
    constexpr int kPieces = kChunks * 16 / kThreads;   // 16-byte pieces of a tile per thread
    constexpr int N = SM::N, KTOT = SM::KTOT, KB = SM::KB;
    extern __shared__ char smem_raw[];
    char *smem = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + SM::MISC);
    uint64_t *mbar_dead = mbar + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM::MISC + 16);
    volatile int *ok_slot = reinterpret_cast<volatile int *>(smem + SM::MISC + 20);
    long long *item = reinterpret_cast<long long *>(smem + SM::MISC + 24);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // chunk row = tensor-memory lane of this thread, and (U pass) which half of the row
    const int cr = tid & (kChunks - 1), half = tid / kChunks;

    if (warp == 0) {
        tmem_alloc(tmem_slot, SM::TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_init(mbar_dead, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    constexpr uint32_t idesc = idesc_tf32_m128(N);
    const int64_t n = hi::plan_count(h.plan, bt);
    const int64_t total = h.plan.tile_pref[n];
    const int Ms = bt.Mstride;
    uint32_t phase = 0;
    int64_t cur_ch = -1;

    // U pass: the tile's x and y rows into XT / YT (zero past tlen)
    auto load_xy = [&](int64_t tstart, int tlen) {
        const bool al = xy_al && ((tstart & 3) == 0);
        for (int q = 0; q < kPieces; ++q) {
            const int id = tid + kThreads * q;
            const int r = id >> 4, j = id & 15;
            const int s0 = r * kL + j * 4;
            const int nv = min(max(tlen - s0, 0), 4);
            const uint32_t dx = sbase + SM::XT + rowp(r, j), dy = sbase + SM::YT + rowp(r, j);
            const float *gx_ = h.x + tstart + s0, *gy_ = h.y + tstart + s0;
            if (al) {
                cp_async16(dx, nv ? (const void *)gx_ : (const void *)h.x, nv * 4);
                cp_async16(dy, nv ? (const void *)gy_ : (const void *)h.y, nv * 4);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    cp_async4(dx + 4 * e, e < nv ? (const void *)(gx_ + e) : (const void *)h.x, e < nv ? 4 : 0);
                    cp_async4(dy + 4 * e, e < nv ? (const void *)(gy_ + e) : (const void *)h.y, e < nv ? 4 : 0);
                }
            }
        }
        cp_async_commit();
    };
    // Tiles are taken in runs of kRun consecutive ones (mostly one channel: the tables
    // are rebuilt only when the channel changes), each tile's channel found with one
    // lookup.  Within a run the next tile's signal tile is copied into the operand while
    // this tile's epilogue runs (also its x and y tiles in the U pass, once this tile's
    // are consumed); not where the U pass's x and y sit over the operand.
    constexpr int kRun = 8;
    constexpr bool kPrefetch = MODE != hi::kU || SM::SEPXY;
    int64_t w = 0, wend = 0;
    bool pre = false;   // this tile's signal (and U: x, y) tiles already copied
    for (;;) {
        if (w >= wend) {
            if (tid == 0) *item = (long long)atomicAdd(h.counter, 1ull);
            __syncthreads();
            w = *item * kRun;
            __syncthreads();   // *item is rewritten at the next run
            if (w >= total) break;
            wend = w + kRun < total ? w + kRun : total;
        }
        const int64_t pos = h.plan.tile_pos[w];
        const int64_t ch = hi::plan_channel(h.plan, pos);
        const Channel c = channel_of(bt, ch);
        const int64_t tile = w - h.plan.tile_pref[pos];
        const int64_t tstart = c.off + tile * kTileSamples;
        const int64_t tl64 = c.len - tile * kTileSamples;
        const int tlen = (int)(tl64 < kTileSamples ? tl64 : kTileSamples);
        const int nch = (tlen + kL - 1) / kL;
        const int64_t slot0 = c.off / kL + ch + tile * kChunks;   // the tile's first chunk slot
        const char *R = h.tabs + (size_t)ch * h.tab_stride;
        // the next tile of the run, whose inputs are copied during this tile's epilogue
        const bool has_next = kPrefetch && w + 1 < wend;
        int64_t ntstart = 0;
        int ntlen = 0;
        if (has_next) {
            const int64_t npos = h.plan.tile_pos[w + 1];
            const Channel nc = channel_of(bt, hi::plan_channel(h.plan, npos));
            const int64_t ntile = w + 1 - h.plan.tile_pref[npos];
            ntstart = nc.off + ntile * kTileSamples;
            const int64_t ntl64 = nc.len - ntile * kTileSamples;
            ntlen = (int)(ntl64 < kTileSamples ? ntl64 : kTileSamples);
        }

        // ---- B operand (the channel's tables), split into TF32 hi | lo ----
        if (ch != cur_ch) {
#pragma unroll 8
            for (int idx = tid; idx < N * KTOT; idx += kThreads) {
                const int nn = idx / KTOT, k = idx % KTOT;
                float v = 0.f;
                if constexpr (MODE == hi::kY) {
                    if (k <= nn) v = reinterpret_cast<const float *>(R + h.tab_g)[nn - k];
                } else {
                    const int n2 = nn & (kL - 1);
                    if (k >= n2)
                        v = reinterpret_cast<const float *>(R + (nn < kL ? Tab::B_G : Tab::B_H))[k - n2];
                }
                float hv, lv;
                split_tf32(v, hv, lv);
                const uint32_t o = (uint32_t)(k >> 5) * SM::BBLK + sw128_off(nn, k & 31);
                *reinterpret_cast<float *>(smem + SM::BHI + o) = hv;
                *reinterpret_cast<float *>(smem + SM::BLO + o) = lv;
            }
            if constexpr (SM::OUT) {
                // the free-response tables: O_L (Y pass), or O^u and O^gx (U pass)
                float *ot = reinterpret_cast<float *>(smem + SM::OT);
                const float *src = reinterpret_cast<const float *>(
                    R + (MODE == hi::kY ? (size_t)h.tab_ol : (size_t)Tab::B_OU));
#pragma unroll 4
                for (int i = tid; i < kL * MB / 4; i += kThreads)
                    reinterpret_cast<float4 *>(ot)[i] = __ldg(reinterpret_cast<const float4 *>(src) + i);
                if constexpr (MODE == hi::kU) {
                    const float *src2 = reinterpret_cast<const float *>(R + Tab::B_OGX);
#pragma unroll 4
                    for (int i = tid; i < kL * MB / 4; i += kThreads)
                        reinterpret_cast<float4 *>(ot + kL * MB)[i] =
                            __ldg(reinterpret_cast<const float4 *>(src2) + i);
                }
            }
            cur_ch = ch;
        }

        // ---- A operand: the signal tile, then (Y, U) the chunk states ----
        if (!pre) {
            pipe::load_tile_async<kThreads>(sbase + SM::AHI, h.sig, tstart, tlen,
                                            sig_al && ((tstart & 3) == 0), tid);
            if constexpr (SM::SEPXY) load_xy(tstart, tlen);
        }
        // (Y, U) this row's chunk state, FP32, for the free response in the epilogue
        float S[SM::OUT ? MB : 1];
        if constexpr (SM::OUT) {
            const float *sv = (MODE == hi::kY ? h.states2 : h.states) + (size_t)(slot0 + cr) * Ms;
            const bool v = cr < nch;
            if (st_al) {   // rows of Mstride floats, 16-byte aligned
#pragma unroll
                for (int m4 = 0; m4 < MB; m4 += 4) {
                    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (v && m4 < c.M) q = __ldg(reinterpret_cast<const float4 *>(sv + m4));
                    S[m4] = q.x;
                    S[m4 + 1] = m4 + 1 < c.M ? q.y : 0.f;
                    S[m4 + 2] = m4 + 2 < c.M ? q.z : 0.f;
                    S[m4 + 3] = m4 + 3 < c.M ? q.w : 0.f;
                }
            } else {
#pragma unroll
                for (int m = 0; m < MB; ++m) S[m] = (v && m < c.M) ? __ldg(sv + m) : 0.f;
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (h.three) {
            for (int id = tid; id < KB * kChunks * 8; id += kThreads) {
                const int kb = id / (kChunks * 8), rem = id % (kChunks * 8);
                const int r = rem >> 3, j = rem & 7;
                const uint32_t o = (uint32_t)kb * kKBlock + (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4));
                const float4 v = *reinterpret_cast<const float4 *>(smem + SM::AHI + o);
                float4 hv, lv;
                split_tf32(v.x, hv.x, lv.x);
                split_tf32(v.y, hv.y, lv.y);
                split_tf32(v.z, hv.z, lv.z);
                split_tf32(v.w, hv.w, lv.w);
                *reinterpret_cast<float4 *>(smem + SM::ALO + o) = lv;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();

        // ---- tensor cores ----
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < KTOT / 8; ++kk) {
                const uint32_t ka = (uint32_t)(kk >> 2) * kKBlock + (kk & 3) * 32;
                const uint32_t kbo = (uint32_t)(kk >> 2) * SM::BBLK + (kk & 3) * 32;
                const uint64_t ahi = sdesc_sw128(sbase + SM::AHI + ka);
                const uint64_t bhi = sdesc_sw128(sbase + SM::BHI + kbo);
                mma_tf32(tmem, ahi, bhi, idesc, kk > 0 ? 1u : 0u);
                if (h.three) {
                    mma_tf32(tmem, ahi, sdesc_sw128(sbase + SM::BLO + kbo), idesc, 1u);
                    mma_tf32(tmem, sdesc_sw128(sbase + SM::ALO + ka), bhi, idesc, 1u);
                }
            }
            mma_commit(mbar);
            bool ok = mbar_wait_bounded(mbar, phase, bt.wait_limit);
            if (ok && bt.stall_drill) ok = mbar_wait_bounded(mbar_dead, 0, bt.wait_limit);
            if (!ok) {
                set_status(bt.status, DFILT_ERR_TIMEOUT);
                mbar_wait_bounded(mbar, phase, kDefaultWaitLimit);   // drain before leaving
            }
            *ok_slot = ok ? 1 : 0;
        }
        phase ^= 1u;
        __syncthreads();
        tc_fence_after();
        if (!*ok_slot) break;
        // the operand is consumed: the next tile's signal goes there now
        if (has_next)
            pipe::load_tile_async<kThreads>(sbase + SM::AHI, h.sig, ntstart, ntlen,
                                            sig_al && ((ntstart & 3) == 0), tid);

        // ---- epilogues (thread = chunk row = TMEM lane) ----
        if constexpr (MODE == hi::kY) {
            char *stag = smem + SM::ALO;   // the operand's low part is consumed (the high part
                                           // receives the next tile)
            const float *ot = reinterpret_cast<const float *>(smem + SM::OT);
#pragma unroll 1
            for (int cb = 0; cb < kL / 16; ++cb) {
                float v[16];
                tmem_ld16(taddr + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float *ol = ot + (cb * 16 + i) * MB;
                    float acc = v[i];
#pragma unroll
                    for (int m4 = 0; m4 < MB; m4 += 4) {   // O_L rows are 16-byte aligned
                        if (m4 < c.M) {   // the state is zero past the channel's order
                            const float4 q = *reinterpret_cast<const float4 *>(ol + m4);
                            acc = fmaf(q.x, S[m4], acc);
                            acc = fmaf(q.y, S[m4 + 1], acc);
                            acc = fmaf(q.z, S[m4 + 2], acc);
                            acc = fmaf(q.w, S[m4 + 3], acc);
                        }
                    }
                    v[i] = acc;
                }
#pragma unroll
                for (int p4 = 0; p4 < 4; ++p4)
                    *reinterpret_cast<float4 *>(stag + rowp(cr, cb * 4 + p4)) =
                        make_float4(v[4 * p4], v[4 * p4 + 1], v[4 * p4 + 2], v[4 * p4 + 3]);
            }
            tc_fence_before();
            __syncthreads();
            const bool al = out_al && ((tstart & 3) == 0);
#pragma unroll 4
            for (int q = 0; q < kPieces; ++q) {
                const int id = tid + kThreads * q;
                const int r = id >> 4, j = id & 15;
                const float4 v = *reinterpret_cast<const float4 *>(stag + rowp(r, j));
                const int s = r * kL + j * 4;
                const int nv = min(max(tlen - s, 0), 4);
                float *g = h.out + tstart + s;
                if (nv == 4 && al) {
                    *reinterpret_cast<float4 *>(g) = v;
                } else {
                    if (nv > 0) g[0] = v.x;
                    if (nv > 1) g[1] = v.y;
                    if (nv > 2) g[2] = v.z;
                    if (nv > 3) g[3] = v.w;
                }
            }
            __syncthreads();
        } else {
            constexpr int KBLK = SM::KBLK, NACC = hi::nacc<MB>();
            const float *ou = reinterpret_cast<const float *>(smem + SM::OT);
            const float *ogx = ou + kL * MB;
            // (1) x and y tiles (rows of 256 bytes) over the consumed operand, unless they
            // were loaded with the signal tile
            if constexpr (!SM::SEPXY) load_xy(tstart, tlen);
            // (2) the adjoint window in tensor memory: u = D + O^u S' over columns
            // 64 .. 128, then S' and zeros (each half of the CTA takes half the columns)
#pragma unroll 1
            for (int cb = 2 * half; cb < 2 * half + 2; ++cb) {
                float v[16];
                tmem_ld16(taddr + kL + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float *o = ou + (cb * 16 + i) * MB;
                    float acc = v[i];
#pragma unroll
                    for (int m4 = 0; m4 < MB; m4 += 4) {
                        if (m4 < c.M) {
                            const float4 q = *reinterpret_cast<const float4 *>(o + m4);
                            acc = fmaf(q.x, S[m4], acc);
                            acc = fmaf(q.y, S[m4 + 1], acc);
                            acc = fmaf(q.z, S[m4 + 2], acc);
                            acc = fmaf(q.w, S[m4 + 3], acc);
                        }
                    }
                    v[i] = acc;
                }
                tmem_st16(taddr + kL + cb * 16, v);
            }
#pragma unroll
            for (int cb = 0; cb < (SM::UEND - 2 * kL + 15) / 16; ++cb) {
                if ((cb & 1) != half) continue;   // static indices into S[]
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = (cb * 16 + i < MB) ? S[cb * 16 + i] : 0.f;
                tmem_st16(taddr + 2 * kL + cb * 16, v);
            }
            tmem_wait_st();
            if constexpr (!SM::SEPXY) cp_async_wait_all();   // x, y over the operand
            __syncthreads();
            const char *xrow = smem + SM::XT, *yrow = smem + SM::YT;
            auto ld16 = [&](const char *base, int j0, float (&v)[16]) {   // samples 4*j0 .. 4*j0+15
#pragma unroll
                for (int p4 = 0; p4 < 4; ++p4) {
                    const float4 q = *reinterpret_cast<const float4 *>(base + rowp(cr, j0 + p4));
                    v[4 * p4] = q.x; v[4 * p4 + 1] = q.y; v[4 * p4 + 2] = q.z; v[4 * p4 + 3] = q.w;
                }
            };
            // (3) lag sums: b-lag k: sum_n u[n+k] x[n] (k = 0..MB), a-lag k: sum_n u[n+1+k] y[n]
            float *red = reinterpret_cast<float *>(smem + SM::RED);
#pragma unroll 1
            for (int kb = 0; kb < KBLK; ++kb) {
                // lag blocks past the channel's orders are skipped (uniform over the CTA):
                // b-lags 16 kb .. need 16 kb <= N, a-lags 16 kb + 1 .. need 16 kb < M
                const bool need_x = 16 * kb <= c.N, need_y = 16 * kb < c.M;
                float acc[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = 0.f;
#pragma unroll 1
                for (int nb = 2 * half; nb < 2 * half + 2 && (need_x || need_y); ++nb) {
                    float xv[16], yv[16], w0[16], w1[16];
                    ld16(yrow, nb * 4, yv);
                    const uint32_t f0 = taddr + kL + 16 * (nb + kb);   // u_ext[16(nb+kb) ..]
                    tmem_ld16(f0, w0);
                    tmem_ld16(f0 + 16, w1);
                    tmem_wait_ld();
#define DFILT_WIN(i) ((i) < 16 ? w0[(i)] : w1[(i) - 16])
                    if (need_x) {
                        ld16(xrow, nb * 4, xv);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                acc[j] = fmaf(DFILT_WIN(q + j), xv[q], acc[j]);
                                acc[16 + j] = fmaf(DFILT_WIN(q + 1 + j), yv[q], acc[16 + j]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                acc[16 + j] = fmaf(DFILT_WIN(q + 1 + j), yv[q], acc[16 + j]);
                        }
                    }
#undef DFILT_WIN
                }
                // warp total of all 32 sums: halving butterfly, lane L ends with sum L
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int i = 0; i < o; ++i) {
                        const bool up = (lane & o) != 0;
                        const float send = up ? acc[i] : acc[i + o];
                        const float keep = up ? acc[i + o] : acc[i];
                        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
                red[(warp * KBLK + kb) * 32 + lane] = acc[0];   // warp = 4 half + quadrant
            }
            // (4) grad_x = D[:, 0:64) + O^gx S', written over this row of the x tile
#pragma unroll 1
            for (int cb = 2 * half; cb < 2 * half + 2; ++cb) {
                float v[16];
                tmem_ld16(taddr + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float *o = ogx + (cb * 16 + i) * MB;
                    float acc = v[i];
#pragma unroll
                    for (int m4 = 0; m4 < MB; m4 += 4) {
                        if (m4 < c.M) {
                            const float4 q = *reinterpret_cast<const float4 *>(o + m4);
                            acc = fmaf(q.x, S[m4], acc);
                            acc = fmaf(q.y, S[m4 + 1], acc);
                            acc = fmaf(q.z, S[m4 + 2], acc);
                            acc = fmaf(q.w, S[m4 + 3], acc);
                        }
                    }
                    v[i] = acc;
                }
#pragma unroll
                for (int p4 = 0; p4 < 4; ++p4)
                    *reinterpret_cast<float4 *>(smem + SM::XT + rowp(cr, cb * 4 + p4)) =
                        make_float4(v[4 * p4], v[4 * p4 + 1], v[4 * p4 + 2], v[4 * p4 + 3]);
            }
            tc_fence_before();
            __syncthreads();
            // the tile's lag sums in a fixed order (warps 0..7)
            for (int i = tid; i < KBLK * 32; i += kThreads) {
                const int kb = i / 32, j = i % 32;
                float v = 0.f;
#pragma unroll
                for (int e = 0; e < kThreads / 32; ++e) v += red[(e * KBLK + kb) * 32 + j];
                const int k = 16 * kb + (j & 15);
                if (j < 16) {
                    if (k <= MB) h.partial[(size_t)w * NACC + k] = v;
                } else if (k < MB) {
                    h.partial[(size_t)w * NACC + MB + 1 + k] = v;
                }
            }
            if (h.out) {
                const bool al = out_al && ((tstart & 3) == 0);
#pragma unroll 4
                for (int q = 0; q < kPieces; ++q) {
                    const int id = tid + kThreads * q;
                    const int r = id >> 4, j = id & 15;
                    const float4 v = *reinterpret_cast<const float4 *>(smem + SM::XT + rowp(r, j));
                    const int s = r * kL + j * 4;
                    const int nv = min(max(tlen - s, 0), 4);
                    float *g = h.out + tstart + s;
                    if (nv == 4 && al) {
                        *reinterpret_cast<float4 *>(g) = v;
                    } else {
                        if (nv > 0) g[0] = v.x;
                        if (nv > 1) g[1] = v.y;
                        if (nv > 2) g[2] = v.z;
                        if (nv > 3) g[3] = v.w;
                    }
                }
            }
            __syncthreads();
            // x and y of the next tile, now that this tile's are consumed
            if constexpr (SM::SEPXY) {
                if (has_next) load_xy(ntstart, ntlen);
            }
        }
        ++w;
        pre = has_next;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, SM::TMEM_COLS);
    }
}

template <int MB, int MODE>
cudaError_t launch_tc(const HiArgs &h, const Batch &bt, int num_sms, cudaStream_t st) {
    using SM = TcSmem<MB, MODE>;
    static_assert(SM::ALLOC <= pipe::kSmemMax, "shared memory budget");
    auto kern = hi_tc_kernel<MB, MODE>;
    static int occ[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::ALLOC);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        // CTAs per SM: shared memory, registers and tensor memory (the persistent CTAs
        // never wait on one another, so a grid larger than what is resident is harmless)
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        int smem_sm = 0, smem_blk = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&smem_blk, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        int o = smem_sm / (int)(SM::ALLOC + smem_blk + fa.sharedSizeBytes);
        const int regs = (fa.numRegs + 7) / 8 * 8;
        const int oreg = regs > 0 ? 65536 / (regs * threads_of<MODE>()) : o;
        o = o < oreg ? o : oreg;
        const int tmem_cap = 512 / (int)SM::TMEM_COLS;
        o = o < tmem_cap ? o : tmem_cap;
        occ[dev] = o < 1 ? 1 : (o > 4 ? 4 : o);
    }
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0 ? 1 : 0; };
    const int xy_al = (h.x && h.y) ? (al(h.x) & al(h.y)) : 0;
    const float *sv = MODE == hi::kY ? h.states2 : h.states;
    const int st_al = (sv && al(sv) && bt.Mstride % 4 == 0) ? 1 : 0;
    kern<<<(unsigned)(num_sms * occ[dev]), threads_of<MODE>(), SM::ALLOC, st>>>(h, bt, al(h.sig),
                                                                      h.out ? al(h.out) : 0, xy_al,
                                                                      st_al); note_launch();
    return cudaGetLastError();
}

}  // namespace

template <int MB>
cudaError_t hi_tc(const HiArgs &h, const Batch &bt, int mode, int num_sms, cudaStream_t st) {
    switch (mode) {
        case hi::kY: return launch_tc<MB, hi::kY>(h, bt, num_sms, st);
        case hi::kU: return launch_tc<MB, hi::kU>(h, bt, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t hi_tc<DFILT_MB>(const HiArgs &, const Batch &, int, int, cudaStream_t);

}  // namespace dfilt
