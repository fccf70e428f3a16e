// Decoupled high-order path, tensor-core tile passes (sm_103a).  Every tile (128 chunks
// x 64 samples of one channel) is independent here, since the chunk states come from
// the scan kernel:
//
//   Y pass             D = X T_g^T              N = 64   -> y = D + O_L S_c
//   U pass             D = G [T_g^a ; T_h^a]^T  N = 128  -> grad_x = D[:, 0:64) + O^gx S'_c
//                                                          and u = D[:, 64:128) + O^u S'_c
// (the lag sums of grad_b, grad_a are formed from u by hi_lag_kernel).
// The free responses O_L S_c, O^u S'_c and O^gx S'_c are added on the CUDA cores in FP32,
// per chunk row: the chunk states of high-order filters are large numbers whose
// combination cancels, and the split-TF32 product (about 21 bits per operand) would cost
// digits there that FP32 FMAs keep.  For the same reason grad_x comes from the impulse
// response of B/A directly, not as B applied to the all-pole adjoint u (which can be far
// larger than grad_x when zeros of B sit near poles of A).
//
// One persistent CTA per SM, warp-specialised so that loads, tensor-core products and
// the FP32 epilogues of different tiles overlap:
//   warps 0-7   epilogue, two groups of four warps taking alternate tiles (group g the
//               tiles k with k mod 2 = g, in tensor-memory accumulator g), so that one
//               group's latencies hide behind the other's work.  Thread = chunk row
//               (tensor-memory lane); lanes l and l^16 of a warp swap halves of their
//               rows so that every shared-memory table load serves two rows.  A group
//               also rebuilds the B operand when its tile starts a new channel (once the
//               previous tile's products are done) and its own copy of the free-response
//               tables when its channel differs from its previous tile's
//   warps 8-10  producer: the tile's samples (one bulk copy of the 16-byte-aligned range
//               around them into linear staging), then the A operand from the staging
//               (the sub-16-byte shift, the swizzle, the TF32 low parts), and the tile's
//               chunk states (cp.async)
//   warp 11     tensor cores: one thread issues the products into accumulator k mod 2
// Tiles are taken in a static order (runs of consecutive tiles, run r on CTA r mod grid),
// which every role walks on its own.  Hand-offs are mbarriers only, each wait bounded:
// a wait that runs out records DFILT_ERR_TIMEOUT and raises a shared abort flag that
// every role polls, so all roles leave their loops (no named barrier is used, so no role
// can be left waiting on another that left).
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
constexpr int kEpiThreads = 256;                      // warps 0-7
constexpr int kProdThreads = 96;                      // warps 8-10
constexpr int kMmaWarp = 11;
constexpr int kThreads = 32 * (kMmaWarp + 1);         // 384: three warps per SM sub-partition
constexpr uint32_t kKBlock = kChunks * 128;           // one 32-wide K block of the A operand
constexpr uint32_t kABytes = 2 * kKBlock;             // one A operand tile (K = 64)

// One tile's position, written by the producer into its stage's slot before the stage
// is published.
struct TcDesc {
    int64_t tstart, slot0, ch;
    int tlen, nch, M;
    int flags;   // kNewB: the channel differs from the previous tile's (B operand rebuilt);
                 // kNewOT: from the tile two before (the group's free-response tables)
};
constexpr int kNewB = 1, kNewOT = 2;
constexpr int kGroupThreads = 128;                    // one epilogue group

template <int MB, int MODE>
struct TcSmem {
    using Tab = ChunkTab<MB>;
    static_assert(MODE == hi::kY || MODE == hi::kU, "tile passes: Y and U");
    static constexpr int N = MODE == hi::kU ? 2 * kL : kL;        // MMA N
    static constexpr int KTOT = kL;
    static constexpr int KB = 2;                                  // K blocks of 32
    static constexpr uint32_t BBLK = (uint32_t)N * 128;           // bytes of one B K block
    static constexpr uint32_t BHI = 0;
    static constexpr uint32_t BLO = KB * BBLK;
    // free-response tables [L][MB] f32 per epilogue group: O_L (Y pass), or O^u then
    // O^gx (U pass)
    static constexpr int NOT = MODE == hi::kU ? 2 : 1;
    static constexpr uint32_t OT = 2 * KB * BBLK;                 // [group][NOT][L][MB]
    static constexpr uint32_t OT_GROUP = (uint32_t)NOT * kL * MB * 4;
    static constexpr uint32_t A0 = (OT + 2 * OT_GROUP + 1023) / 1024 * 1024;
    // the A operand (hi = the raw FP32 words, lo = the TF32 remainders), one buffer
    static constexpr uint32_t AHI = A0;
    static constexpr uint32_t ALO = A0 + kABytes;
    // linear staging of a tile's samples, from the 16-byte boundary at or before its
    // first sample (one bulk copy per tile); two stages where shared memory allows
    static constexpr uint32_t RAWB = (uint32_t)kTileSamples * 4 + 128;
    static constexpr uint32_t RAW0 = ALO + kABytes;
    static constexpr uint32_t MISC_BYTES = 512;
    static constexpr int NRAW = RAW0 + 2 * RAWB + MISC_BYTES + 1024 <= pipe::kSmemMax ? 2 : 1;
    static constexpr uint32_t AEND = RAW0 + NRAW * RAWB;
    // the tiles' chunk states, two stages of 128 rows (padded rows: conflict-free float4
    // reads), where shared memory allows; else the epilogue reads them from global memory
    static constexpr int SROW = MB + 4;
    static constexpr uint32_t SBYTES = (uint32_t)kChunks * SROW * 4;
    static constexpr bool SSTAGE = AEND + 2 * SBYTES + MISC_BYTES + 1024 <= pipe::kSmemMax;
    static constexpr uint32_t S0 = AEND;
    static constexpr uint32_t MISC = SSTAGE ? S0 + 2 * SBYTES : AEND;
    static constexpr uint32_t BYTES = MISC + MISC_BYTES;
    static constexpr uint32_t ALLOC = BYTES + 1024;
    static constexpr uint32_t TMEM_COLS = 2 * N;                  // two accumulators
};

// Store 16 consecutive outputs to g (g % 4 floats == D): scalar head, float4 body, tail.
template <int D>
__device__ __forceinline__ void st16(float *g, const float (&v)[16]) {
    constexpr int H = (4 - D) & 3, Q = (16 - H - D) / 4;
#pragma unroll
    for (int j = 0; j < H; ++j) g[j] = v[j];
#pragma unroll
    for (int q = 0; q < Q; ++q)
        *reinterpret_cast<float4 *>(g + H + 4 * q) =
            make_float4(v[H + 4 * q], v[H + 4 * q + 1], v[H + 4 * q + 2], v[H + 4 * q + 3]);
#pragma unroll
    for (int j = 0; j < D; ++j) g[16 - D + j] = v[16 - D + j];
}
// The first n (may be <= 0) of 16 outputs.
__device__ __forceinline__ void store16(float *g, const float (&v)[16], int n) {
    if (n >= 16) {
        switch ((int)((reinterpret_cast<uintptr_t>(g) >> 2) & 3)) {
            case 0: st16<0>(g, v); break;
            case 1: st16<1>(g, v); break;
            case 2: st16<2>(g, v); break;
            default: st16<3>(g, v); break;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < n) g[j] = v[j];
    }
}

// Wait for an mbarrier phase with the thread suspended in hardware (up to kSuspendNs per
// call) rather than polling: every thread of the epilogue and producer warps waits, and
// polls from that many threads would saturate the shared-memory pipe the epilogue needs.
constexpr uint32_t kSuspendNs = 1000;
__device__ __forceinline__ bool mbar_wait_susp(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// The static tile order of this CTA: runs of `run` consecutive tiles, run r on CTA
// r mod gridDim.x.  Every role walks the same sequence.
struct TileWalk {
    int64_t total, run, r, w, wend;
    __device__ TileWalk(int64_t total_, int64_t run_) : total(total_), run(run_) {
        r = blockIdx.x;
        w = r * run;
        wend = w + run < total ? w + run : total;
    }
    // the next tile, or -1
    __device__ int64_t next() {
        if (w >= wend) {
            r += gridDim.x;
            w = r * run;
            wend = w + run < total ? w + run : total;
            if (w >= total) return -1;
        }
        return w < total ? w++ : -1;
    }
};

template <int MB, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    hi_tc_kernel(HiArgs h, Batch bt, int sig_al, int st_al) {
    using Tab = ChunkTab<MB>;
    using SM = TcSmem<MB, MODE>;
    constexpr int N = SM::N, KTOT = SM::KTOT;
    extern __shared__ char smem_raw[];
    char *smem = smem_align1024(smem_raw);
    const uint32_t sbase = smem_u32(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + SM::MISC);   // [2] A operand ready (96)
    uint64_t *mma_done = full + 2;    // [2] accumulator ready, A operand consumed (commit)
    uint64_t *acc_free = full + 4;    // [2] group done with its accumulator (128)
    uint64_t *s_free = full + 6;      // [2] group has read its stage's states and slot (128)
    uint64_t *tab_full = full + 8;    // B operand of a new channel written (128)
    uint64_t *ot_full = full + 9;     // [2] a group's free-response tables written (128)
    uint64_t *raw_full = full + 11;   // [2] staging filled (bulk copy bytes, or 96 cp.async)
    uint64_t *raw_free = full + 13;   // [2] staging converted (96)
    uint64_t *dead = full + 15;       // stall drill: nothing arrives
    uint64_t *drain = full + 16;      // tensor-core work drained before exit
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM::MISC + 144);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + SM::MISC + 148);
    TcDesc *slot = reinterpret_cast<TcDesc *>(smem + SM::MISC + 160);   // [4], tile k in k & 3
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == kMmaWarp) {
        tmem_alloc(tmem_slot, SM::TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full[s], kProdThreads);
            mbar_init(&mma_done[s], 1);
            mbar_init(&acc_free[s], kGroupThreads);
            mbar_init(&s_free[s], kGroupThreads);
            mbar_init(&ot_full[s], kGroupThreads);
            mbar_init(&raw_full[s], sig_al ? 1 : kProdThreads);
            mbar_init(&raw_free[s], kProdThreads);
        }
        mbar_init(tab_full, kGroupThreads);
        mbar_init(dead, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t n = hi::plan_count(h.plan, bt);
    const int64_t total = h.plan.tile_pref[n];
    // about ten runs per CTA; each run keeps its channel's tables over its tiles
    int64_t run = total / ((int64_t)gridDim.x * 10);
    run = run < 4 ? 4 : (run > 32 ? 32 : run);
    const int Ms = bt.Mstride;
    // bounded wait (the poll budget counts 64 polls per suspended call, about a second in
    // all by default); on timeout or a peer's abort every role leaves its loop
    auto wait = [&](uint64_t *bar, int64_t completion) -> bool {
        const uint32_t par = (uint32_t)(completion & 1);
        for (long long it = 0; it < bt.wait_limit; it += 64) {
            if (mbar_wait_susp(bar, par)) return true;
            if (*abort_flag) return false;
        }
        set_status(bt.status, DFILT_ERR_TIMEOUT);
        *abort_flag = 1;
        return false;
    };

    if (warp >= 8 && warp < kMmaWarp) {
        // ============================ producer ==============================
        const int pt = tid - kEpiThreads;
        const float *sv_src = MODE == hi::kY ? h.states2 : h.states;
        constexpr int NRAW = SM::NRAW;
        // tile k: its slot, its chunk states (cp.async, one group per tile) and the fill
        // of its staging (one bulk copy from the 16-byte boundary at or before the first
        // sample up to the last boundary inside the tile; the at most 3 samples past that
        // are read from global memory by the conversion)
        auto issue = [&](int64_t k, const TcDesc &d) -> bool {
            const int rs = (int)(k % NRAW);
            if (k >= 2 && !wait(&s_free[k & 1], (k - 2) >> 1)) return false;
            if (k >= NRAW && !wait(&raw_free[rs], (k - NRAW) / NRAW)) return false;
            if (pt == 0) slot[k & 3] = d;
            if constexpr (SM::SSTAGE) {
                // rows pt, pt + 96 of the tile's chunk states (zero past the order and the
                // tile)
                const int s = (int)(k & 1);
                for (int row = pt; row < kChunks; row += kProdThreads) {
                    const uint32_t dst = sbase + SM::S0 + (uint32_t)s * SM::SBYTES + (uint32_t)row * SM::SROW * 4;
                    const bool v = row < d.nch;
                    const float *src = sv_src + (size_t)(d.slot0 + (v ? row : 0)) * Ms;
                    if (st_al) {
#pragma unroll
                        for (int m4 = 0; m4 < MB; m4 += 4) {
                            const int nv = v ? min(max(d.M - m4, 0), 4) : 0;
                            cp_async16(dst + 4 * m4, nv ? (const void *)(src + m4) : (const void *)sv_src, nv * 4);
                        }
                    } else {
#pragma unroll 4
                        for (int m = 0; m < MB; ++m) {
                            const bool e = v && m < d.M;
                            cp_async4(dst + 4 * m, e ? (const void *)(src + m) : (const void *)sv_src, e ? 4 : 0);
                        }
                    }
                }
            }
            const int64_t a0 = d.tstart & ~(int64_t)3;
            const int n_al = (int)(((d.tstart + d.tlen) & ~(int64_t)3) - a0);   // multiple of 4
            const uint32_t raw = sbase + SM::RAW0 + (uint32_t)rs * SM::RAWB;
            if (sig_al) {
                if (pt == 0) {
                    mbar_arrive_expect_tx(&raw_full[rs], (uint32_t)n_al * 4);
                    if (n_al > 0) bulk_load(raw, h.sig + a0, (uint32_t)n_al * 4, &raw_full[rs]);
                }
            } else {   // (a base address off the 16-byte grid: word copies)
                for (int i = pt; i < n_al; i += kProdThreads) cp_async4(raw + 4 * i, h.sig + a0 + i, 4);
                cp_async_mbar_arrive_noinc(&raw_full[rs]);
            }
            cp_async_commit();
            return true;
        };
        // tile j: the A operand from its staging once the products of tile j - 1 are done,
        // then publish it
        auto finish = [&](int64_t j, const TcDesc &d, bool last) -> bool {
            const int rs = (int)(j % NRAW);
            if (!wait(&raw_full[rs], j / NRAW)) return false;
            if (last) cp_async_wait_all();
            else cp_async_wait_1();   // this thread's state rows of tile j
            if (j >= 1 && !wait(&mma_done[(j - 1) & 1], (j - 1) >> 1)) return false;
            const float *raw = reinterpret_cast<const float *>(smem + SM::RAW0 + (uint32_t)rs * SM::RAWB);
            const int64_t a0 = d.tstart & ~(int64_t)3;
            const int dd = (int)(d.tstart - a0);
            const int n_al = (int)(((d.tstart + d.tlen) & ~(int64_t)3) - a0);
            // batches of four pieces: every load of a batch before its stores (stores to
            // shared memory would otherwise order the next piece's loads after them)
            constexpr int NPC = (2048 + kProdThreads - 1) / kProdThreads;   // pieces per thread
#pragma unroll 1
            for (int q0 = 0; q0 < NPC; q0 += 4) {
                float4 q0v[4], q1v[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int id = pt + kProdThreads * (q0 + b);
                    const int i0 = id < 2048 ? (id >> 4) * kL + (id & 15) * 4 : 0;
                    q0v[b] = *reinterpret_cast<const float4 *>(raw + i0);
                    q1v[b] = *reinterpret_cast<const float4 *>(raw + i0 + 4);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int id = pt + kProdThreads * (q0 + b);
                    if (id >= 2048) break;
                    const int r = id >> 4, j16 = id & 15;
                    const int i0 = r * kL + j16 * 4;   // first sample of the piece
                    const float4 qa = q0v[b], qb = q1v[b];
                    float v[4];
                    switch (dd) {   // uniform over the tile
                        case 0: v[0] = qa.x; v[1] = qa.y; v[2] = qa.z; v[3] = qa.w; break;
                        case 1: v[0] = qa.y; v[1] = qa.z; v[2] = qa.w; v[3] = qb.x; break;
                        case 2: v[0] = qa.z; v[1] = qa.w; v[2] = qb.x; v[3] = qb.y; break;
                        default: v[0] = qa.w; v[1] = qb.x; v[2] = qb.y; v[3] = qb.z; break;
                    }
                    if (i0 + 4 > d.tlen || dd + i0 + 4 > n_al) {   // the tile's ragged end
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int i = i0 + e;
                            v[e] = i >= d.tlen ? 0.f : (dd + i < n_al ? v[e] : __ldg(h.sig + d.tstart + i));
                        }
                    }
                    const uint32_t o = pipe::op_piece(r, j16);
                    *reinterpret_cast<float4 *>(smem + SM::AHI + o) = make_float4(v[0], v[1], v[2], v[3]);
                    if (h.three) {
                        float4 hv, lv;
                        split_tf32(v[0], hv.x, lv.x);
                        split_tf32(v[1], hv.y, lv.y);
                        split_tf32(v[2], hv.z, lv.z);
                        split_tf32(v[3], hv.w, lv.w);
                        *reinterpret_cast<float4 *>(smem + SM::ALO + o) = lv;
                    }
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&raw_free[rs]);
            mbar_arrive(&full[j & 1]);
            return true;
        };
        TileWalk walk(total, run);
        int64_t k = 0;
        bool ok = true;
        int64_t w_prev = -1, pos = -1, ch = -1, ch1 = -1, ch2 = -1;   // ch1, ch2: tiles k-1, k-2
        Channel c{};
        TcDesc dprev{};
        for (;;) {
            if (*abort_flag) break;
            const int64_t w = walk.next();
            if (w < 0) break;
            // the tile's position (tiles of one channel are consecutive)
            if (w != w_prev + 1 || pos < 0 || w >= h.plan.tile_pref[pos + 1]) {
                pos = h.plan.tile_pos[w];
                ch = hi::plan_channel(h.plan, pos, bt);
                c = channel_of(bt, ch);
            }
            w_prev = w;
            const int64_t tile = w - h.plan.tile_pref[pos];
            TcDesc d;
            d.tstart = c.off + tile * kTileSamples;
            const int64_t tl = c.len - tile * kTileSamples;
            d.tlen = (int)(tl < kTileSamples ? tl : kTileSamples);
            d.nch = (d.tlen + kL - 1) / kL;
            d.slot0 = c.off / kL + ch + tile * kChunks;
            d.ch = ch;
            d.M = c.M;
            d.flags = (ch != ch1 ? kNewB : 0) | (ch != ch2 ? kNewOT : 0);
            ch2 = ch1;
            ch1 = ch;
            // debug build: a tile that fails its index checks becomes empty (no sample or
            // state is read or written)
            if (!hi::dbg_range_ok(bt, d.tstart, d.tlen, d.slot0, d.nch)) {
                d.tlen = 0;
                d.nch = 0;
            }
            // one staging buffer: convert the previous tile before refilling it
            if (NRAW == 1 && k >= 1 && !finish(k - 1, dprev, true)) {
                ok = false;
                break;
            }
            if (!issue(k, d)) {
                ok = false;
                break;
            }
            if (NRAW == 2 && k >= 1 && !finish(k - 1, dprev, false)) {
                ok = false;
                break;
            }
            dprev = d;
            ++k;
        }
        if (ok && k >= 1 && !*abort_flag) finish(k - 1, dprev, true);
        cp_async_wait_all();
    } else if (warp == kMmaWarp) {
        // ============================ tensor cores ==========================
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32_m128(N);
            TileWalk walk(total, run);
            int64_t k = 0, nt = 0;
            bool issued = false;
            for (;;) {
                if (*abort_flag) break;
                if (walk.next() < 0) break;
                const int s = (int)(k & 1);
                if (!wait(&full[s], k >> 1)) break;
                if (slot[k & 3].flags & kNewB) {   // an epilogue group rebuilds B first
                    if (!wait(tab_full, nt)) break;
                    ++nt;
                }
                if (k >= 2 && !wait(&acc_free[s], (k - 2) >> 1)) break;
                if (bt.stall_drill) {   // timeout drill: a barrier nothing signals
                    wait(dead, 0);
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)s * N;
#pragma unroll
                for (int kk = 0; kk < KTOT / 8; ++kk) {
                    const uint32_t ka = (uint32_t)(kk >> 2) * kKBlock + (kk & 3) * 32;
                    const uint32_t kbo = (uint32_t)(kk >> 2) * SM::BBLK + (kk & 3) * 32;
                    const uint64_t ahi = sdesc_sw128(sbase + SM::AHI + ka);
                    const uint64_t bhi = sdesc_sw128(sbase + SM::BHI + kbo);
                    mma_tf32(d_tmem, ahi, bhi, idesc, kk > 0 ? 1u : 0u);
                    if (h.three) {
                        mma_tf32(d_tmem, ahi, sdesc_sw128(sbase + SM::BLO + kbo), idesc, 1u);
                        mma_tf32(d_tmem, sdesc_sw128(sbase + SM::ALO + ka), bhi, idesc, 1u);
                    }
                }
                mma_commit(&mma_done[s]);
                issued = true;
                ++k;
            }
            // every tensor-core operation issued completes before the CTA leaves
            if (issued) {
                mma_commit(drain);
                mbar_wait_bounded(drain, 0, kDefaultWaitLimit);
            }
        }
        __syncwarp();
    } else {
        // ============================ epilogue ==============================
        const int g = warp >> 2;                           // group: tiles k = g mod 2
        const int gt = tid & (kGroupThreads - 1);          // = chunk row = TMEM lane
        const int cr = gt;
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)g * N;
        constexpr bool kPair = MB <= 32;
        const bool lower = lane < 16;
        float *ot = reinterpret_cast<float *>(smem + SM::OT + (uint32_t)g * SM::OT_GROUP);
        TileWalk walk(total, run);
        int64_t k = 0, not_ = 0;
        for (;; ++k) {
            if (*abort_flag) break;
            if (walk.next() < 0) break;
            if ((int)(k & 1) != g) continue;
            if (!wait(&full[g], k >> 1)) break;
            const TcDesc d = slot[k & 3];
            const char *R = h.tabs + (size_t)d.ch * h.tab_stride;
            if (d.flags & kNewB) {
                // new channel: once the previous tile's products are done, the B operand
                if (k >= 1 && !wait(&mma_done[g ^ 1], (k - 1) >> 1)) break;
                constexpr int PER = N * KTOT / kGroupThreads, CH = 32;
#pragma unroll 1
                for (int q0 = 0; q0 < PER; q0 += CH) {
                    float vals[CH];
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        const int idx = gt + kGroupThreads * (q0 + q);
                        const int nn = idx / KTOT, kx = idx % KTOT;
                        float v = 0.f;
                        if constexpr (MODE == hi::kY) {
                            if (kx <= nn) v = __ldg(reinterpret_cast<const float *>(R + h.tab_g) + (nn - kx));
                        } else {
                            const int n2 = nn & (kL - 1);
                            if (kx >= n2)
                                v = __ldg(reinterpret_cast<const float *>(R + (nn < kL ? Tab::B_G : Tab::B_H)) +
                                          (kx - n2));
                        }
                        vals[q] = v;
                    }
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        const int idx = gt + kGroupThreads * (q0 + q);
                        const int nn = idx / KTOT, kx = idx % KTOT;
                        float hv, lv;
                        split_tf32(vals[q], hv, lv);
                        const uint32_t o = (uint32_t)(kx >> 5) * SM::BBLK + sw128_off(nn, kx & 31);
                        *reinterpret_cast<float *>(smem + SM::BHI + o) = hv;
                        *reinterpret_cast<float *>(smem + SM::BLO + o) = lv;
                    }
                }
                fence_proxy_async_smem();
                mbar_arrive(tab_full);
            }
            if (d.flags & kNewOT) {
                // the group's free-response tables, once it is done with its previous tile
                if (k >= 2 && !wait(&acc_free[g], (k - 2) >> 1)) break;
                const float4 *src = reinterpret_cast<const float4 *>(
                    R + (MODE == hi::kY ? (size_t)h.tab_ol : (size_t)Tab::B_OU));
#pragma unroll
                for (int i = gt; i < kL * MB / 4; i += kGroupThreads)
                    reinterpret_cast<float4 *>(ot)[i] = __ldg(src + i);
                if constexpr (MODE == hi::kU) {
                    const float4 *src2 = reinterpret_cast<const float4 *>(R + Tab::B_OGX);
#pragma unroll
                    for (int i = gt; i < kL * MB / 4; i += kGroupThreads)
                        reinterpret_cast<float4 *>(ot + kL * MB)[i] = __ldg(src2 + i);
                }
                mbar_arrive(&ot_full[g]);
                if (!wait(&ot_full[g], not_)) break;
                ++not_;
            }
            // this row's chunk state and (paired lanes) that of row cr ^ 16
            float S[MB], S2[kPair ? MB : 1];
            if constexpr (SM::SSTAGE) {
                const float *sb = reinterpret_cast<const float *>(smem + SM::S0 + (uint32_t)g * SM::SBYTES);
#pragma unroll
                for (int m4 = 0; m4 < MB; m4 += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(sb + cr * SM::SROW + m4);
                    S[m4] = q.x;
                    S[m4 + 1] = q.y;
                    S[m4 + 2] = q.z;
                    S[m4 + 3] = q.w;
                }
                if constexpr (kPair) {
#pragma unroll
                    for (int m4 = 0; m4 < MB; m4 += 4) {
                        const float4 q = *reinterpret_cast<const float4 *>(sb + (cr ^ 16) * SM::SROW + m4);
                        S2[m4] = q.x;
                        S2[m4 + 1] = q.y;
                        S2[m4 + 2] = q.z;
                        S2[m4 + 3] = q.w;
                    }
                }
            } else {
                // from global memory: 16-byte loads where the rows are aligned
                const float *sv = (MODE == hi::kY ? h.states2 : h.states) + (size_t)d.slot0 * Ms;
                auto load_row = [&](int row, float (&dst)[MB]) {
                    const bool v = row < d.nch;
                    const float *src = sv + (size_t)(v ? row : 0) * Ms;
                    if (st_al) {
#pragma unroll
                        for (int m4 = 0; m4 < MB; m4 += 4) {
                            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (v && m4 < d.M) q = __ldg(reinterpret_cast<const float4 *>(src + m4));
                            dst[m4] = q.x;
                            dst[m4 + 1] = m4 + 1 < d.M ? q.y : 0.f;
                            dst[m4 + 2] = m4 + 2 < d.M ? q.z : 0.f;
                            dst[m4 + 3] = m4 + 3 < d.M ? q.w : 0.f;
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < MB; ++m) dst[m] = (v && m < d.M) ? __ldg(src + m) : 0.f;
                    }
                };
                load_row(cr, S);
                if constexpr (kPair) load_row(cr ^ 16, S2);
            }
            mbar_arrive(&s_free[g]);
            if (!wait(&mma_done[g], k >> 1)) break;
            tc_fence_after();
            // outputs: Y: y from columns 0..63 with O_L; U: grad_x from 0..63 with O^gx,
            // u from 64..127 with O^u.  A shared-memory load of a table row costs the same
            // whether its 16 bytes serve one row or several, so up to order 32 each table
            // load serves two rows: in each step lanes l and l^16 swap one 16-column block
            // of their rows (shuffles) and each finishes one block for both rows.  Order
            // 64 keeps one row per thread (two rows' states would not fit in registers).
#pragma unroll 1
            for (int which = 0; which < SM::NOT; ++which) {
                float *dst = which ? h.ubuf : h.out;
                if (!dst) continue;   // (grad_x not wanted)
                const float *O = MODE == hi::kY ? ot : (which ? ot : ot + kL * MB);
                const uint32_t col = lane_base + (uint32_t)(which * kL);
#pragma unroll 1
                for (int p = 0; p < 2; ++p) {
                    if constexpr (kPair) {
                        // lower lanes finish block p, upper lanes block p + 2, of both rows
                        float va[16], vb[16];
                        tmem_ld16(col + (uint32_t)(16 * p), va);
                        tmem_ld16(col + (uint32_t)(16 * p + 32), vb);
                        tmem_wait_ld();
                        const int cb = lower ? p : p + 2;
                        float own[16], oth[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            own[j] = lower ? va[j] : vb[j];
                            oth[j] = __shfl_xor_sync(0xffffffffu, lower ? vb[j] : va[j], 16);
                        }
                        // four columns at a time: eight independent FMA chains (each output
                        // still sums its terms in the order m = 0, 1, ...)
#pragma unroll
                        for (int i0 = 0; i0 < 16; i0 += 4) {
                            const float *o = O + (cb * 16 + i0) * MB;
                            float a0[4], a1[4];
#pragma unroll
                            for (int ii = 0; ii < 4; ++ii) {
                                a0[ii] = own[i0 + ii];
                                a1[ii] = oth[i0 + ii];
                            }
#pragma unroll
                            for (int m4 = 0; m4 < MB; m4 += 4) {   // rows are 16-byte aligned
                                if (m4 < d.M) {   // the state is zero past the channel's order
#pragma unroll
                                    for (int ii = 0; ii < 4; ++ii) {
                                        const float4 q = *reinterpret_cast<const float4 *>(o + ii * MB + m4);
                                        a0[ii] = fmaf(q.x, S[m4], a0[ii]);
                                        a1[ii] = fmaf(q.x, S2[m4], a1[ii]);
                                        a0[ii] = fmaf(q.y, S[m4 + 1], a0[ii]);
                                        a1[ii] = fmaf(q.y, S2[m4 + 1], a1[ii]);
                                        a0[ii] = fmaf(q.z, S[m4 + 2], a0[ii]);
                                        a1[ii] = fmaf(q.z, S2[m4 + 2], a1[ii]);
                                        a0[ii] = fmaf(q.w, S[m4 + 3], a0[ii]);
                                        a1[ii] = fmaf(q.w, S2[m4 + 3], a1[ii]);
                                    }
                                }
                            }
#pragma unroll
                            for (int ii = 0; ii < 4; ++ii) {
                                own[i0 + ii] = a0[ii];
                                oth[i0 + ii] = a1[ii];
                            }
                        }
                        const int s0 = cr * kL + cb * 16, s1 = (cr ^ 16) * kL + cb * 16;
                        store16(dst + d.tstart + s0, own, d.tlen - s0);
                        store16(dst + d.tstart + s1, oth, d.tlen - s1);
                    } else {
#pragma unroll 1
                        for (int cb = 2 * p; cb < 2 * p + 2; ++cb) {
                            float v[16];
                            tmem_ld16(col + (uint32_t)(cb * 16), v);
                            tmem_wait_ld();
#pragma unroll
                            for (int i0 = 0; i0 < 16; i0 += 8) {   // eight chains at a time
                                const float *o = O + (cb * 16 + i0) * MB;
#pragma unroll
                                for (int m4 = 0; m4 < MB; m4 += 4) {
                                    if (m4 < d.M) {
#pragma unroll
                                        for (int ii = 0; ii < 8; ++ii) {
                                            const float4 q = *reinterpret_cast<const float4 *>(o + ii * MB + m4);
                                            v[i0 + ii] = fmaf(q.x, S[m4], v[i0 + ii]);
                                            v[i0 + ii] = fmaf(q.y, S[m4 + 1], v[i0 + ii]);
                                            v[i0 + ii] = fmaf(q.z, S[m4 + 2], v[i0 + ii]);
                                            v[i0 + ii] = fmaf(q.w, S[m4 + 3], v[i0 + ii]);
                                        }
                                    }
                                }
                            }
                            const int s0 = cr * kL + cb * 16;
                            store16(dst + d.tstart + s0, v, d.tlen - s0);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_free[g]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, SM::TMEM_COLS);
    }
}

template <int MB, int MODE>
cudaError_t launch_tc(const HiArgs &h, const Batch &bt, int num_sms, cudaStream_t st) {
    using SM = TcSmem<MB, MODE>;
    static_assert(SM::ALLOC <= pipe::kSmemMax, "shared memory budget");
    static_assert(SM::TMEM_COLS <= 512, "tensor memory");
    static_assert(160 + sizeof(TcDesc) * 4 <= SM::MISC_BYTES, "misc area");
    static_assert((SM::N * SM::KTOT / kGroupThreads) % 32 == 0, "B operand rebuild in chunks of 32");
    auto kern = hi_tc_kernel<MB, MODE>;
    static bool attr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::ALLOC);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0 ? 1 : 0; };
    const float *sv = MODE == hi::kY ? h.states2 : h.states;
    const int st_al = (sv && al(sv) && bt.Mstride % 4 == 0) ? 1 : 0;
    // one CTA per SM (more shared memory than half an SM holds)
    kern<<<(unsigned)num_sms, kThreads, SM::ALLOC, st>>>(h, bt, al(h.sig), st_al); note_launch();
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
