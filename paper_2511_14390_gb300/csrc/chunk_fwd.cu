// Chunked forward on the 5th-generation tensor cores (sm_103a).
//
// A CTA owns whole channels (taken from a work counter) and walks each channel's
// tiles of 128 chunks x 64 samples in time order, carrying the TDF-II state across
// tiles.  Per tile:
//   1. cp.async the 8192-sample signal tile into shared memory in the 128-byte
//      swizzled K-major layout (row = chunk, K = sample within the chunk), split it
//      into TF32 hi/lo parts;
//   2. one thread issues tcgen05.mma: D[128 x (L+MPAD)] = X [T_g | R_L]^T with the
//      3-term split (hi*hi + hi*lo + lo*hi), FP32 accumulation in tensor memory.
//      Columns 0..L-1 of row c are chunk c's zero-state response, columns L.. its
//      zero-state end state E_c (Sec. 3.2 operator at chunk granularity);
//   3. the 128 threads (thread c <-> TMEM lane c <-> chunk c) scan the chunk states
//      S_{c+1} = Abar S_c + E_c: a Hillis-Steele scan in FP32 over precomputed powers
//      Abar^(2^k) for low orders, or a work-efficient serial scan in FP64 (one warp)
//      where FP32 powers lose stability (high-order filters);
//   4. epilogue: y = D + O_L S_c, staged through shared memory and stored coalesced;
//      the chunk entry states go to `saved` for the backward's recomputation of y.
#include <cstring>

#include "chunk_pipe.cuh"

#ifndef DFILT_MB
#error "compile once per state bucket with -DDFILT_MB=<2|4|8|16|32|64>"
#endif

namespace dfilt {

namespace {

constexpr int kThreads = 128;
constexpr uint32_t kSmemMax = 232448;               // opt-in shared memory per block
constexpr uint32_t kTileBytes = kChunks * kL * 4;   // 32 KB
constexpr uint32_t kKBlock = kChunks * 128;         // one 32-wide K block of the A operand

template <int MB, bool F64>
struct FwdSmem {
    using Tab = ChunkTab<MB>;
    static constexpr int NM = Tab::NFWD;
    static constexpr uint32_t AHI = 0;
    static constexpr uint32_t ALO = AHI + kTileBytes;
    static constexpr uint32_t BHI = ALO + kTileBytes;
    static constexpr uint32_t BLO = BHI + NM * 256;
    static constexpr uint32_t OL = BLO + NM * 256;
    static constexpr uint32_t SCAN = OL + kL * MB * 4;
    static constexpr uint32_t MISC = (SCAN + (uint32_t)Tab::scan_bytes(F64) + 15) / 16 * 16;
    // misc block: mbarrier (8) | tmem base (4) | channel (8) | flag (4) | drill mbarrier (8) |
    // S_in (MB doubles) | serial-scan state (2 x MB double words)
    static constexpr uint32_t ST = MISC + 48 + MB * 8;
    static constexpr uint32_t BYTES = ST + 2 * MB * 8;
    static constexpr uint32_t ALLOC = BYTES + 1024;   // slack for 1024-byte alignment
};

// Load samples [start, start+n) of src into the swizzled A tile at `dst` (2 K blocks),
// zero-filling past n.  Thread t of NT handles the 16-byte pieces t, t+NT, ...
template <int NT = kThreads>
__device__ __forceinline__ void load_tile(uint32_t dst, const float *src, int64_t start, int n,
                                          bool al16) {
#pragma unroll 4
    for (int q = 0; q < 2048 / NT; ++q) {
        const int id = threadIdx.x + NT * q;
        const int r = id >> 4, j16 = id & 15;
        const uint32_t d = dst + (j16 >> 3) * kKBlock + r * 128 + ((((j16 & 7) ^ (r & 7))) << 4);
        const int s = r * kL + j16 * 4;
        const int nv = min(max(n - s, 0), 4);
        const float *g = src + start + s;
        if (al16) {
            cp_async16(d, nv ? (const void *)g : (const void *)src, nv * 4);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                cp_async4(d + 4 * e, e < nv ? (const void *)(g + e) : (const void *)src, e < nv ? 4 : 0);
        }
    }
    cp_async_commit();
}

// Split this thread's pieces of the A tile into TF32 hi (in place) and lo (at +lo_off).
template <int NT = kThreads>
__device__ __forceinline__ void split_tile(char *smem, uint32_t a_off, uint32_t lo_off, bool three) {
#pragma unroll 4
    for (int q = 0; q < 2048 / NT; ++q) {
        const int id = threadIdx.x + NT * q;
        const int r = id >> 4, j16 = id & 15;
        const uint32_t o = a_off + (j16 >> 3) * kKBlock + r * 128 + ((((j16 & 7) ^ (r & 7))) << 4);
        float4 v = *reinterpret_cast<float4 *>(smem + o);
        float4 h, l;
        split_tf32(v.x, h.x, l.x);
        split_tf32(v.y, h.y, l.y);
        split_tf32(v.z, h.z, l.z);
        split_tf32(v.w, h.w, l.w);
        *reinterpret_cast<float4 *>(smem + o) = h;
        if (three) *reinterpret_cast<float4 *>(smem + o + lo_off) = l;
    }
}

// Store n samples of the staged tile (row c = chunk c, 256-byte rows, 16-byte pieces
// XOR-swizzled by row) to dst[start ..].
template <int NT = kThreads>
__device__ __forceinline__ void store_tile(float *dst, int64_t start, int n, const char *stag,
                                           bool al16) {
#pragma unroll 4
    for (int q = 0; q < 2048 / NT; ++q) {
        const int id = threadIdx.x + NT * q;
        const int r = id >> 4, j = id & 15;
        const float4 v = *reinterpret_cast<const float4 *>(stag + r * 256 + ((j ^ (r & 15)) << 4));
        const int s = r * kL + j * 4;
        const int nv = min(max(n - s, 0), 4);
        float *g = dst + start + s;
        if (nv == 4 && al16) {
            *reinterpret_cast<float4 *>(g) = v;
        } else {
            if (nv > 0) g[0] = v.x;
            if (nv > 1) g[1] = v.y;
            if (nv > 2) g[2] = v.z;
            if (nv > 3) g[3] = v.w;
        }
    }
}

template <int MB>
__device__ __forceinline__ void matvec_f32(const float *P, const float (&v)[MB], float (&out)[MB]) {
#pragma unroll
    for (int i = 0; i < MB; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < MB; ++j) acc = fmaf(P[i * MB + j], v[j], acc);
        out[i] = acc;
    }
}

template <int MB, bool F64>
__global__ void __launch_bounds__(kThreads, 1)
    chunk_fwd_kernel(const float *__restrict__ x, const float *__restrict__ zi,
                     float *__restrict__ y, float *__restrict__ saved, const char *__restrict__ tabs,
                     unsigned long long *__restrict__ counter, Batch bt, int three, int x_al,
                     int y_al) {
    using Tab = ChunkTab<MB>;
    using SM = FwdSmem<MB, F64>;
    constexpr int NM = SM::NM;
    extern __shared__ char smem_raw[];
    char *smem = smem_align1024(smem_raw);
    const uint32_t sbase = smem_u32(smem);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + SM::MISC);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM::MISC + 8);
    int64_t *ch_slot = reinterpret_cast<int64_t *>(smem + SM::MISC + 16);
    int *flag_slot = reinterpret_cast<int *>(smem + SM::MISC + 24);
    double *sin_buf = reinterpret_cast<double *>(smem + SM::MISC + 48);
    float *sOL = reinterpret_cast<float *>(smem + SM::OL);
    const float *sP = reinterpret_cast<const float *>(smem + SM::SCAN);
    const float2 *sAt = reinterpret_cast<const float2 *>(smem + SM::SCAN);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tmem_alloc(tmem_slot, 128);
        tmem_relinquish();
    }
    uint64_t *mbar_dead = reinterpret_cast<uint64_t *>(smem + SM::MISC + 32);   // never signalled (timeout drill)
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_init(mbar_dead, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool alive = true;
    const size_t rec = bt.fwd_stride ? (size_t)bt.fwd_stride : Tab::fwd_rec(F64);
    constexpr uint32_t idesc = idesc_tf32_m128(NM);

    while (alive) {
        if (tid == 0) {
            int64_t cw = -1;
            if (!work_channel(bt, (int64_t)atomicAdd(counter, 1ull), &cw)) cw = -1;
            *ch_slot = cw;
        }
        __syncthreads();
        const int64_t ch = *ch_slot;
        if (ch < 0) break;
        const Channel c = channel_of(bt, ch);
        const char *R = tabs + (size_t)ch * rec;
        // ---- per-channel operand tables ----
        {
            const float *g = reinterpret_cast<const float *>(R + Tab::F_G);
            const float *RL = reinterpret_cast<const float *>(R + Tab::F_RL);
            for (int idx = tid; idx < NM * kL; idx += kThreads) {
                const int i = idx / kL, k = idx % kL;
                float v = 0.f;
                if (i < kL) v = k <= i ? g[i - k] : 0.f;
                else if (i < kL + MB) v = RL[(i - kL) * kL + k];
                float h, l;
                split_tf32(v, h, l);
                const uint32_t o = (k >> 5) * (NM * 128) + sw128_off(i, k & 31);
                *reinterpret_cast<float *>(smem + SM::BHI + o) = h;
                *reinterpret_cast<float *>(smem + SM::BLO + o) = l;
            }
            const float *OL = reinterpret_cast<const float *>(R + Tab::F_OL);
            for (int idx = tid; idx < kL * MB; idx += kThreads) sOL[idx] = OL[idx];
            const float4 *src = reinterpret_cast<const float4 *>(R + Tab::F_SCAN);
            float4 *dst = reinterpret_cast<float4 *>(smem + SM::SCAN);
            for (int idx = tid; idx < (int)(Tab::scan_bytes(F64) / 16); idx += kThreads) dst[idx] = src[idx];
            if (tid < MB) sin_buf[tid] = (zi && tid < c.M) ? (double)zi[ch * bt.Mstride + tid] : 0.0;
        }
        fence_proxy_async_smem();
        __syncthreads();

        // per-thread carried state for the FP32 scan; the serial scan carries its
        // double-word state in shared memory (st[0..MB))
        float Sin[MB];
        float2 *st = reinterpret_cast<float2 *>(smem + SM::ST);
#pragma unroll
        for (int m = 0; m < MB; ++m) Sin[m] = (float)sin_buf[m];
        if (F64 && tid < MB) st[tid] = make_float2((float)sin_buf[tid], 0.f);
        const int64_t ntiles = (c.len + kTileSamples - 1) / kTileSamples;
        const int64_t chunk_base = c.off / kL + ch;

        for (int64_t t = 0; t < ntiles; ++t) {
            const int64_t tstart = c.off + t * kTileSamples;
            const int tlen = (int)(c.len - t * kTileSamples < kTileSamples ? c.len - t * kTileSamples : kTileSamples);
            const int nch = (tlen + kL - 1) / kL;
            const bool al = x_al && ((tstart & 3) == 0);
            load_tile(sbase + SM::AHI, x, tstart, tlen, al);
            cp_async_wait_all();
            split_tile(smem, SM::AHI, SM::ALO - SM::AHI, three != 0);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int s = 0; s < kL / 8; ++s) {
                    const uint32_t ka = (s >> 2) * kKBlock + (s & 3) * 32;
                    const uint32_t kb = (s >> 2) * (NM * 128) + (s & 3) * 32;
                    const uint64_t ahi = sdesc_sw128(sbase + SM::AHI + ka);
                    const uint64_t bhi = sdesc_sw128(sbase + SM::BHI + kb);
                    mma_tf32(tmem, ahi, bhi, idesc, s > 0 ? 1u : 0u);
                    if (three) {
                        const uint64_t alo = sdesc_sw128(sbase + SM::ALO + ka);
                        const uint64_t blo = sdesc_sw128(sbase + SM::BLO + kb);
                        mma_tf32(tmem, ahi, blo, idesc, 1u);
                        mma_tf32(tmem, alo, bhi, idesc, 1u);
                    }
                }
                mma_commit(mbar);
                bool ok = mbar_wait_bounded(mbar, phase, bt.wait_limit);
                if (ok && bt.stall_drill) ok = mbar_wait_bounded(mbar_dead, 0, bt.wait_limit);
                if (!ok) {
                    set_status(bt.status, DFILT_ERR_TIMEOUT);
                    // drain: the MMAs still own tensor memory; wait for them before leaving
                    mbar_wait_bounded(mbar, phase, kDefaultWaitLimit);
                }
                *flag_slot = ok ? 1 : 0;
            }
            phase ^= 1u;
            __syncthreads();
            tc_fence_after();
            if (!*flag_slot) {
                alive = false;
                break;
            }

            // ---- chunk end states E_c (TMEM columns L .. L+MB) ----
            float E[MB];
            {
#pragma unroll
                for (int cb = 0; cb < Tab::MPAD / 16; ++cb) {
                    float v[16];
                    tmem_ld16(taddr + kL + cb * 16, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (cb * 16 + i < MB) E[cb * 16 + i] = v[i];
                }
            }
            float S[MB];   // state entering this thread's chunk
            float *xbuf = reinterpret_cast<float *>(smem + SM::ALO);   // A tile is free now
            if constexpr (!F64) {
                // Two-level scan.  (1) warp-local inclusive Hillis-Steele over the warp's 32
                // chunks: W_c = sum_{j=32w..c} Abar^(c-j) E_j;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int d = 1 << k;
                    float prev[MB];
#pragma unroll
                    for (int m = 0; m < MB; ++m) prev[m] = __shfl_up_sync(0xffffffffu, E[m], d);
                    if (lane >= d) {
                        float add[MB];
                        matvec_f32<MB>(sP + k * MB * MB, prev, add);
#pragma unroll
                        for (int m = 0; m < MB; ++m) E[m] += add[m];
                    }
                }
                // (2) carries: C_0 = S_in, C_{w+1} = Abar^32 C_w + W_{32w+31} (state entering
                // chunk 32w); C_4 leaves the tile;
                if (lane == 31) {
#pragma unroll
                    for (int m = 0; m < MB; ++m) xbuf[warp * MB + m] = E[m];
                }
                __syncthreads();
                float C[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) C[m] = Sin[m];
                for (int ww = 0; ww < kChunks / 32; ++ww) {
                    if (ww == warp) {
#pragma unroll
                        for (int m = 0; m < MB; ++m) S[m] = C[m];
                    }
                    float w2[MB];
                    matvec_f32<MB>(sP + 5 * MB * MB, C, w2);
#pragma unroll
                    for (int m = 0; m < MB; ++m) C[m] = w2[m] + xbuf[ww * MB + m];
                }
#pragma unroll
                for (int m = 0; m < MB; ++m) Sin[m] = C[m];
                // (3) entry state of chunk c = 32w + l: Abar^l C_w + W_{c-1}
                float v[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) v[m] = S[m];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if ((lane >> k) & 1) {
                        float w2[MB];
                        matvec_f32<MB>(sP + k * MB * MB, v, w2);
#pragma unroll
                        for (int m = 0; m < MB; ++m) v[m] = w2[m];
                    }
                }
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    const float wprev = __shfl_up_sync(0xffffffffu, E[m], 1);
                    S[m] = v[m] + (lane > 0 ? wprev : 0.f);
                }
                __syncthreads();
            } else {
                // serial scan S_{c+1} = Abar S_c + E_c by the whole CTA, state carried in
                // double words
                float *sbuf = reinterpret_cast<float *>(smem + SM::AHI);
#pragma unroll
                for (int m = 0; m < MB; ++m) xbuf[tid * MB + m] = E[m];
                __syncthreads();
                pipe::dw_scan_group<MB>(sAt, st, xbuf, sbuf, nch, false, tid, [] { __syncthreads(); });
                if ((nch & 1) && tid < MB) st[tid] = st[MB + tid];   // outgoing state to st[0]
                __syncthreads();
#pragma unroll
                for (int m = 0; m < MB; ++m) S[m] = tid < nch ? sbuf[tid * MB + m] : 0.f;
                __syncthreads();
            }

            // ---- save the chunk entry states for the backward ----
            if (saved && tid < nch) {
                float *dst = saved + (size_t)(chunk_base + t * kChunks + tid) * bt.Mstride;
#pragma unroll
                for (int m = 0; m < MB; ++m)
                    if (m < c.M) dst[m] = S[m];
            }

            // ---- epilogue: y = D + O_L S, staged in the (free) A_hi region ----
            char *stag = smem + SM::AHI;
#pragma unroll 1
            for (int cb = 0; cb < kL / 16; ++cb) {
                float v[16];
                tmem_ld16(taddr + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float *ol = sOL + (cb * 16 + i) * MB;
                    float acc = v[i];
#pragma unroll
                    for (int m = 0; m < MB; ++m) acc = fmaf(ol[m], S[m], acc);
                    v[i] = acc;
                }
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int j = cb * 4 + p;
                    *reinterpret_cast<float4 *>(stag + tid * 256 + ((j ^ (tid & 15)) << 4)) =
                        make_float4(v[4 * p], v[4 * p + 1], v[4 * p + 2], v[4 * p + 3]);
                }
            }
            tc_fence_before();
            __syncthreads();
            store_tile(y, tstart, tlen, stag, y_al && ((tstart & 3) == 0));
            __syncthreads();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 128);
    }
}

template <int MB, bool F64>
cudaError_t launch_fwd_t(const float *x, const float *zi, float *y, float *saved, const char *tabs,
                         unsigned long long *counter,
                         const Batch &bt, int three, int num_sms, cudaStream_t st) {
    using SM = FwdSmem<MB, F64>;
    auto kern = chunk_fwd_kernel<MB, F64>;
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
        int smem_sm = 0, smem_blk = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&smem_blk, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        // CTAs per SM that the shared-memory budget allows (tensor memory allows 4 x 128
        // columns; the register budget is checked by the occupancy query)
        int o = smem_sm / (int)(SM::ALLOC + smem_blk);
        int oq = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oq, kern, kThreads, SM::ALLOC);
        if (e != cudaSuccess) return e;
        if (oq > 0 && oq < o) o = oq;
        occ[dev] = o < 1 ? 1 : (o > 2 ? 2 : o);   // tensor memory: 128 columns per CTA
    }
    const int64_t slots = (int64_t)num_sms * occ[dev];
    const int64_t grid = bt.B < slots ? bt.B : slots;
    const int x_al = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    const int y_al = (reinterpret_cast<uintptr_t>(y) & 15) == 0;
    kern<<<(unsigned)grid, kThreads, SM::ALLOC, st>>>(x, zi, y, saved, tabs, counter, bt, three, x_al, y_al); note_launch();
    return cudaGetLastError();
}


// ===========================================================================
// Shared-memory layout of the pipelined forward: NST signal-tile stages (the raw tile
// is the TF32 hi operand; its lo part lives in TMEM), one y staging buffer, and two
// per-channel table slots (B operand hi | lo, O_L, scan block, S_in).
// ===========================================================================

// (layouts are also instantiated only to test whether they fit, so some of their
// members go unreferenced)
#pragma nv_diag_suppress 177
template <int MB, bool F64, int NST>
struct PipeSmem {
    using Tab = ChunkTab<MB>;
    static constexpr int NM = Tab::NFWD;
    static constexpr uint32_t XS0 = 0;                              // NST x tiles
    static constexpr uint32_t YS = NST * kTileBytes;                // y staging
    static constexpr uint32_t TAB0 = YS + kTileBytes;
    // per table slot: B hi | B lo | O_L | scan block | S_in (doubles)
    static constexpr uint32_t T_BHI = 0;
    static constexpr uint32_t T_BLO = T_BHI + NM * 256;
    static constexpr uint32_t T_OL = T_BLO + NM * 256;
    static constexpr uint32_t T_SCAN = T_OL + kL * MB * 4;
    static constexpr uint32_t T_SIN = (T_SCAN + (uint32_t)Tab::scan_bytes(F64) + 15) / 16 * 16;
    static constexpr uint32_t TSLOT = (T_SIN + MB * 8 + 1023) / 1024 * 1024;
    static constexpr uint32_t MISC = TAB0 + 2 * TSLOT;
};

struct TileDesc {
    int64_t ch;        // channel (-1: none)
    int64_t tstart;    // first sample (packed index)
    int64_t chunk0;    // first chunk's index in `saved`
    int32_t tlen;      // valid samples in the tile
    int32_t tab;       // table slot
    int32_t first;     // first tile of its channel
    int32_t M;         // channel order (for saved states)
    int32_t last;      // last tile of its channel
};

// ===========================================================================
// Warp-specialised forward (state buckets whose double-buffered layout fits).
//
// Roles (384 threads), decoupled by mbarriers; signal tiles in NST shared-memory
// stages (s = i % NST), TMEM operand slots alternating (i & 1), accumulators in a ring
// of NA (i % NA; three 80-column accumulators where they fit beside the operand slots):
//   warps 0-2, 8-11  converters: fetch work; build per-channel tables (double-buffered by
//              channel parity); signal tiles arrive NST-1 ahead (TMA tensor load into
//              the 128-byte-swizzled operand layout, or cp.async when the layout has no
//              chunk-aligned rows); warps 8-11 write the TF32 operand (the raw words as
//              hi, x - trunc(x) as lo) into TMEM operand slot i&1 once MMA(i-2) is done
//                                                   -> full[s]; the stage is then free
//   warp 3     MMA issuer: full[s], tmem_free -> tcgen05.mma (A from TMEM, the B operand
//              from shared memory) into TMEM accumulator i%NA -> mma_done (commit)
//   warps 4-7  epilogue: mma_done -> chunk-state scan, y = D + O_L S, saved states; y
//              staged in the y buffer in the operand layout and written by a TMA tensor
//              store (full tiles) or plain stores     -> tmem_free
// ===========================================================================
// The forward's epilogue needs few registers, so this pipeline runs 12 warps: the
// converters are warps 0-2 and 8-11 (224 threads), the MMA issuer warp 3 and the
// epilogue warps 4-7 (one per TMEM lane quarter).
constexpr int kConvThreads = 224;
constexpr int kFwdThreads = 384;
using pipe::kEpiWarp0;
using pipe::kMmaWarp;
using pipe::kNamedConv;
using pipe::kNamedEpi;
using pipe::named_sync;

template <int MB, bool F64, int NST>
struct WsSmem {
    using P = PipeSmem<MB, F64, NST>;
    static constexpr uint32_t MISC = P::MISC;
    // barriers: full[3] (unused)[3] load[3] mma_done[3] tmem_free[3] tab_free[2] dead
    // drain (19 of 20 slots)
    static constexpr int NBAR = 20;
    static constexpr uint32_t M_BAR = MISC;
    static constexpr uint32_t M_TMEM = MISC + NBAR * 8;
    static constexpr uint32_t M_ABORT = M_TMEM + 4;
    static constexpr uint32_t M_OK = M_TMEM + 8;      // converter (2) / epilogue broadcast words
    static constexpr uint32_t M_WT = M_TMEM + 32;
    static constexpr uint32_t M_RING = (M_WT + 4 * MB * 4 + 15) / 16 * 16;
    static constexpr int RING = 8;
    static constexpr uint32_t BYTES = M_RING + RING * 48;
    static constexpr uint32_t ALLOC = BYTES + 1024;
};
// three signal-tile stages (two tiles of loads in flight) where they fit, else two
template <int MB, bool F64>
constexpr int fwd_stages() {
    return WsSmem<MB, F64, 3>::ALLOC <= kSmemMax ? 3 : 2;
}
#pragma nv_diag_default 177

using pipe::op_piece;

template <int MB, bool F64, int NST>
__global__ void __launch_bounds__(kFwdThreads, 1)
    chunk_fwd_ws_kernel(const float *__restrict__ x, const float *__restrict__ zi,
                        float *__restrict__ y, float *__restrict__ saved,
                        const char *__restrict__ tabs, unsigned long long *__restrict__ counter,
                        Batch bt, int three, int x_al, int y_al, int use_tma,
                        const __grid_constant__ CUtensorMap tmx,
                        const __grid_constant__ CUtensorMap tmy) {
    using Tab = ChunkTab<MB>;
    using PS = PipeSmem<MB, F64, NST>;
    using SM = WsSmem<MB, F64, NST>;
    constexpr int NM = PS::NM;
    constexpr int LA = NST - 1;          // tiles loaded ahead of the one being converted
    constexpr int RING = SM::RING;
    extern __shared__ char smem_raw[];
    char *smem = smem_align1024(smem_raw);
    const uint32_t sbase = smem_u32(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SM::M_BAR);
    uint64_t *full = bars + 0, *load_bar = bars + 6, *mma_done = bars + 9,
             *tmem_free = bars + 12, *tab_free = bars + 15, *dead = bars + 17, *drain = bars + 18;
    // accumulators: NA of ACOLS columns below the operand slots (columns 256 ..)
    constexpr int NA = 3 * NM <= 256 ? 3 : 2;
    constexpr uint32_t ACOLS = NA == 3 ? (uint32_t)NM : 128u;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM::M_TMEM);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + SM::M_ABORT);
    // decision flags written by one thread and read by its role after a named barrier;
    // each decision point has its own word, so that a late reader never sees the value
    // of a later point (the roles must leave their loops at the same point)
    volatile int *conv_ok = reinterpret_cast<volatile int *>(smem + SM::M_OK);
    volatile int *epi_ok = reinterpret_cast<volatile int *>(smem + SM::M_OK + 8);
    float *wt = reinterpret_cast<float *>(smem + SM::M_WT);
    TileDesc *ring = reinterpret_cast<TileDesc *>(smem + SM::M_RING);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < SM::NBAR; ++i) mbar_init(&bars[i], (i >= 9 && i < 12) ? 2 : 1);   // mma_done: commit + arrive
        *abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const size_t rec = bt.fwd_stride ? (size_t)bt.fwd_stride : Tab::fwd_rec(F64);
    auto stage_hi = [&](int s) { return (uint32_t)(PS::XS0 + s * kTileBytes); };
    auto tslot = [&](int p) { return (uint32_t)(PS::TAB0 + p * PS::TSLOT); };
    // TMEM columns of stage s's A_lo (128 lanes = chunks x 64 columns = samples)
    auto ahi_col = [&](int p) { return (uint32_t)(256 + 128 * p); };
    auto alo_col = [&](int p) { return (uint32_t)(256 + 128 * p + 64); };
    // bounded wait by one thread; on timeout (or a peer's abort) raise the abort flag
    auto wait1 = [&](uint64_t *bar, uint32_t parity) -> bool {
        for (long long it = 0; it < bt.wait_limit; ++it) {
            if (mbar_try_wait(bar, parity)) return true;
            if ((it & 63) == 63) {
                if (*abort_flag) return false;
                __nanosleep(32);
            }
        }
        set_status(bt.status, DFILT_ERR_TIMEOUT);
        *abort_flag = 1;
        return false;
    };

    if (warp < kMmaWarp || warp >= 8) {
        // ============================ converters ============================
        const int ct = warp < kMmaWarp ? tid : tid - 160;   // 0..kConvThreads-1
        int64_t cur_ch = -1, cur_t = 0, cur_nt = 0, cur_off = 0, cur_len = 0;
        int cur_M = 1, ch_seq = -1;
        // thread 0: describe the next tile into `d` (published to the ring by the caller)
        auto next_desc = [&](TileDesc &d) {
            while (cur_ch < 0 || cur_t >= cur_nt) {
                int64_t c;
                if (!work_channel(bt, (int64_t)atomicAdd(counter, 1ull), &c)) {
                    d.ch = -1;
                    return;
                }
                const Channel cc = channel_of(bt, c);
                cur_ch = c;
                cur_t = 0;
                cur_off = cc.off;
                cur_len = cc.len;
                cur_M = cc.M;
                cur_nt = (cc.len + kTileSamples - 1) / kTileSamples;
                if (cur_nt == 0) continue;
                ++ch_seq;
            }
            d.ch = cur_ch;
            d.tstart = cur_off + cur_t * kTileSamples;
            d.tlen = (int)(cur_len - cur_t * kTileSamples < kTileSamples ? cur_len - cur_t * kTileSamples
                                                                         : kTileSamples);
            d.chunk0 = cur_off / kL + cur_ch + cur_t * kChunks;
            d.tab = ch_seq & 1;
            d.first = cur_t == 0;
            d.M = cur_M;
            ++cur_t;
            d.last = cur_t == cur_nt;
        };
        // all converters: per-channel tables into slot d.tab (column-parallel expansion
        // of the Toeplitz block: thread handles column k, half h of the rows)
        auto build_tables = [&](const TileDesc &d) {
            const char *R = tabs + (size_t)d.ch * rec;
            const float *__restrict__ g = reinterpret_cast<const float *>(R + Tab::F_G);
            const float *__restrict__ RL = reinterpret_cast<const float *>(R + Tab::F_RL);
            char *T = smem + tslot(d.tab);
            // work item = (column k, half of the Toeplitz rows; the second half also
            // writes the end-state rows R_L and the zero padding)
            for (int item = ct; item < 128; item += kConvThreads) {
                const int k = item & 63, h = item >> 6;
                float gv[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int r = 32 * h + q;
                    gv[q] = r >= k ? __ldg(g + (r - k)) : 0.f;
                }
                float rv[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) rv[m] = h ? __ldg(RL + m * kL + k) : 0.f;
                const uint32_t kb = (k >> 5) * (NM * 128);
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int r = 32 * h + q;
                    float hv, lv;
                    split_tf32(gv[q], hv, lv);
                    const uint32_t o = kb + sw128_off(r, k & 31);
                    *reinterpret_cast<float *>(T + PS::T_BHI + o) = hv;
                    *reinterpret_cast<float *>(T + PS::T_BLO + o) = lv;
                }
                if (h) {
#pragma unroll
                    for (int r = kL; r < NM; ++r) {
                        const float v = r < kL + MB ? rv[r - kL] : 0.f;
                        float hv, lv;
                        split_tf32(v, hv, lv);
                        const uint32_t o = kb + sw128_off(r, k & 31);
                        *reinterpret_cast<float *>(T + PS::T_BHI + o) = hv;
                        *reinterpret_cast<float *>(T + PS::T_BLO + o) = lv;
                    }
                }
            }
            const float4 *OL = reinterpret_cast<const float4 *>(R + Tab::F_OL);
            float4 *sOL = reinterpret_cast<float4 *>(T + PS::T_OL);
            for (int idx = ct; idx < kL * MB / 4; idx += kConvThreads) sOL[idx] = __ldg(OL + idx);
            const float4 *src = reinterpret_cast<const float4 *>(R + Tab::F_SCAN);
            float4 *dst = reinterpret_cast<float4 *>(T + PS::T_SCAN);
            for (int idx = ct; idx < (int)(Tab::scan_bytes(F64) / 16); idx += kConvThreads) dst[idx] = __ldg(src + idx);
            double *sin = reinterpret_cast<double *>(T + PS::T_SIN);
            if (ct < MB) sin[ct] = (zi && ct < d.M) ? (double)zi[d.ch * bt.Mstride + ct] : 0.0;
            fence_proxy_async_smem();   // B is read by the tensor cores
        };
        // tile i's signal into stage s's hi slot (TMA by thread 0, or cp.async by all)
        auto issue_load = [&](const TileDesc &d, int s) {
            if (use_tma) {
                if (ct == 0) {
                    mbar_arrive_expect_tx(&load_bar[s], kTileBytes);
                    const int row = (int)(d.tstart / kL);
                    tma_load_3d(sbase + stage_hi(s), &tmx, 0, 0, row, &load_bar[s]);
                    tma_load_3d(sbase + stage_hi(s) + kKBlock, &tmx, 0, 1, row, &load_bar[s]);
                }
            } else {
                pipe::load_tile_async<kConvThreads>(sbase + stage_hi(s), x, d.tstart, d.tlen,
                                                    x_al && ((d.tstart & 3) == 0), ct);
            }
        };

        // TF32 operand of stage s's tile into TMEM operand slot p (warps 8-11, one TMEM
        // lane quarter each, thread = chunk row): the raw word as A_hi (the tensor cores
        // truncate a TF32 operand to its upper 19 bits) and x - trunc(x) as A_lo; samples
        // past the tile's end are zero (a TMA load may bring in the next channel's)
        auto a_to_tmem = [&](int n, int s, int p) {
            const int q = warp & 3;
            const int r = 32 * q + lane;
            const char *hi = smem + stage_hi(s);
            const int nv = n - r * kL;   // valid samples of this row
            const uint32_t lrow = (uint32_t)(32 * q) << 16;
            auto rows = [&](auto full) {   // full: every sample of the row is valid (no masking)
#pragma unroll
                for (int cb = 0; cb < kL / 16; ++cb) {
                    float vh[16], vl[16];
#pragma unroll
                    for (int p4 = 0; p4 < 4; ++p4) {
                        const int j16 = cb * 4 + p4;
                        const float4 v = *reinterpret_cast<const float4 *>(hi + op_piece(r, j16));
                        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float xv = (decltype(full)::value || 4 * j16 + c < nv) ? e[c] : 0.f;
                            float h;
                            split_tf32(xv, h, vl[4 * p4 + c]);
                            vh[4 * p4 + c] = xv;
                        }
                    }
                    tmem_st16(tmem + lrow + ahi_col(p) + cb * 16, vh);
                    if (three) tmem_st16(tmem + lrow + alo_col(p) + cb * 16, vl);
                }
            };
            // warp-uniform choice: tcgen05.st is a warp-collective instruction
            if (__all_sync(0xffffffffu, nv >= kL)) rows(pipe::BoolC<true>{});
            else rows(pipe::BoolC<false>{});
            tmem_wait_st();
            tc_fence_before();
        };

        // prologue: tiles 0 .. LA-1 described, their tables built and loads issued
        if (ct == 0) {
            for (int j = 0; j < LA; ++j) {
                TileDesc dj;
                next_desc(dj);
                ring[j] = dj;
            }
        }
        named_sync(kNamedConv, kConvThreads);
        int64_t issued_upto = -1;   // last tile whose load this thread has issued
        for (int j = 0; j < LA; ++j) {
            const TileDesc dj = ring[j];
            if (dj.ch < 0) break;
            if (dj.first) build_tables(dj);   // channel slots 0 / 1: not in use yet
            issue_load(dj, j);
            issued_upto = j;
        }
        for (int64_t i = 0;; ++i) {
            const int s = (int)(i % NST);
            const uint32_t ph = (uint32_t)((i / NST) & 1);
            const TileDesc d = ring[i & (RING - 1)];
            if (d.ch < 0) {
                if (ct == 0) mbar_arrive(&full[s]);   // end marker for the MMA warp
                break;
            }
            // (1) tile i landed in stage s; TMEM operand slot i&1 free once MMA(i-2), its
            //     previous reader, is done
            if (ct == 0) {
                bool ok = true;
                if (use_tma) ok = wait1(&load_bar[s], ph);
                if (ok && i >= 2) ok = wait1(&mma_done[(i - 2) % NA], (uint32_t)(((i - 2) / NA) & 1));
                conv_ok[0] = ok ? 1 : 0;
            }
            if (!use_tma) {
                if (issued_upto > i) cp_async_wait_1();
                else cp_async_wait_all();
            }
            named_sync(kNamedConv, kConvThreads);
            if (!conv_ok[0]) break;
            // (2) the operand into TMEM; the stage is free from here on
            if (warp >= 8) {
                tc_fence_after();
                a_to_tmem(d.tlen, s, (int)(i & 1));
            }
            named_sync(kNamedConv, kConvThreads);
            if (ct == 0) mbar_arrive(&full[s]);
            // (3) tile i+LA: descriptor, tables of a new channel, load into its stage (tile
            //     i-1's, converted in the previous iteration).  Ring slots are reused 8 tiles
            //     apart; through the waits above the epilogue has started tile i-4.
            if (ct == 0) {
                TileDesc nd;
                next_desc(nd);
                bool ok = true;
                if (nd.ch >= 0 && nd.first) {
                    // slot nd.tab was last used two channels ago
                    const int seq = ch_seq;
                    if (seq >= 2) ok = wait1(&tab_free[nd.tab], (uint32_t)(((seq >> 1) - 1) & 1));
                }
                ring[(i + LA) & (RING - 1)] = nd;
                conv_ok[1] = ok ? 1 : 0;
            }
            named_sync(kNamedConv, kConvThreads);
            if (!conv_ok[1]) break;
            const TileDesc dn = ring[(i + LA) & (RING - 1)];
            if (dn.ch >= 0) {
                // the load first: its stage is free already, and the tables (global
                // reads of the channel's record) are needed only when its MMA runs
                issue_load(dn, (int)((i + LA) % NST));
                issued_upto = i + LA;
                if (dn.first) build_tables(dn);
            }
        }
    } else if (warp == kMmaWarp) {
        // ============================ MMA issuer ============================
        bool issued = false;
        for (int64_t i = 0;; ++i) {
            const int s = (int)(i % NST);        // signal-tile stage
            const int tb_ = (int)(i & 1);          // TMEM operand slot
            const int ab = (int)(i % NA);          // TMEM accumulator
            const uint32_t par = (uint32_t)((i / NA) & 1);
            int ok = 1;
            if (lane == 0) ok = wait1(&full[s], (uint32_t)((i / NST) & 1)) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            const TileDesc d = ring[i & (RING - 1)];
            // TMEM buffer free (epilogue done with tile i-2); the end marker waits too,
            // or its arrivals could complete a second phase of mma_done before the
            // epilogue has observed tile i-2's (a parity wait cannot tell them apart)
            if (lane == 0 && i >= NA) ok = wait1(&tmem_free[ab], par ^ 1u) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            if (d.ch < 0) {
                if (lane == 0) {
                    mbar_arrive(&mma_done[ab]);   // end marker for the epilogue (2 arrivals)
                    mbar_arrive(&mma_done[ab]);
                }
                break;
            }
            if (lane == 0) {
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)ab * ACOLS;
                const uint32_t tb = tslot(d.tab);
#pragma unroll
                for (int kk = 0; kk < kL / 8; ++kk) {
                    // T_g is lower triangular: samples 8kk .. 8kk+7 reach outputs n >= 8kk
                    // only, so this K step covers B rows (and D columns) from n0 on; the
                    // R_L rows behind T_g are dense and always included
                    const int n0 = 16 * (kk / 2);
                    const uint32_t kb = (kk >> 2) * (NM * 128) + (kk & 3) * 32 + n0 * 128;
                    const uint32_t idn = idesc_tf32_m128(NM - n0);
                    const uint32_t dk = d_tmem + (uint32_t)n0;
                    const uint32_t ahi = tmem + ahi_col(tb_) + 8 * kk;
                    const uint64_t bhi = sdesc_sw128(sbase + tb + PS::T_BHI + kb);
                    mma_tf32_tmem_a(dk, ahi, bhi, idn, kk > 0 ? 1u : 0u);
                    if (three) {
                        const uint64_t blo = sdesc_sw128(sbase + tb + PS::T_BLO + kb);
                        mma_tf32_tmem_a(dk, ahi, blo, idn, 1u);
                        mma_tf32_tmem_a(dk, tmem + alo_col(tb_) + 8 * kk, bhi, idn, 1u);
                    }
                }
                mma_commit(&mma_done[ab]);
                mbar_arrive(&mma_done[ab]);   // orders the descriptor reads before the epilogue's
            }
            issued = true;
            if (bt.stall_drill) {
                if (lane == 0) wait1(dead, 0);   // timeout drill: a barrier nothing signals
                __syncwarp();
                break;
            }
        }
        // drain: every tensor-core operation this warp issued completes before exit
        if (lane == 0 && issued) {
            mma_commit(drain);
            mbar_wait_bounded(drain, 0, kDefaultWaitLimit);
        }
        __syncwarp();
    } else {
        // ============================ epilogue ==============================
        const int et = tid - kEpiWarp0 * 32;   // 0..127 = chunk = TMEM lane
        const int ew = warp - kEpiWarp0;       // lane quarter
        const uint32_t lane_off = (uint32_t)(ew * 32) << 16;
        float Sin[MB];
        // the serial scan's double-word state [2][MB], in the warp-total area (which only
        // the FP32 scan uses)
        float2 *st = reinterpret_cast<float2 *>(wt);
#pragma unroll
        for (int m = 0; m < MB; ++m) Sin[m] = 0.f;
        for (int64_t i = 0;; ++i) {
            const int s = (int)(i % NA);           // TMEM accumulator
            const uint32_t par = (uint32_t)((i / NA) & 1);
            if (et == 0) *epi_ok = wait1(&mma_done[s], par) ? 1 : 0;
            named_sync(kNamedEpi, 128);
            if (!*epi_ok) break;
            tc_fence_after();
            const TileDesc pv = ring[i & (RING - 1)];
            if (pv.ch < 0) break;
            const char *T = smem + tslot(pv.tab);
            const float *sOL = reinterpret_cast<const float *>(T + PS::T_OL);
            const float *sP = reinterpret_cast<const float *>(T + PS::T_SCAN);
            const float2 *sAt = reinterpret_cast<const float2 *>(T + PS::T_SCAN);
            const double *sin = reinterpret_cast<const double *>(T + PS::T_SIN);
            const int nch = (pv.tlen + kL - 1) / kL;
            const uint32_t taddr = tmem + lane_off + (uint32_t)s * ACOLS;
            if (pv.first) {
#pragma unroll
                for (int m = 0; m < MB; ++m) Sin[m] = (float)sin[m];
                if (F64 && et < MB) st[et] = make_float2((float)sin[et], 0.f);
            }
            float E[MB];
#pragma unroll
            for (int cb = 0; cb < Tab::MPAD / 16; ++cb) {
                float v[16];
                tmem_ld16(taddr + kL + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (cb * 16 + q < MB) E[cb * 16 + q] = v[q];
            }
            float S[MB];
            // the y buffer: serial-scan scratch, then y staging (free once the bulk store of
            // the previous tile has read it)
            char *lo = smem + PS::YS;
            if constexpr (!F64) {
                // two-level scan: warp-local Hillis-Steele, then carries across the 4 warps
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int dd = 1 << k;
                    float prev[MB];
#pragma unroll
                    for (int m = 0; m < MB; ++m) prev[m] = __shfl_up_sync(0xffffffffu, E[m], dd);
                    if (lane >= dd) {
                        float add[MB];
                        matvec_f32<MB>(sP + k * MB * MB, prev, add);
#pragma unroll
                        for (int m = 0; m < MB; ++m) E[m] += add[m];
                    }
                }
                if (lane == 31) {
#pragma unroll
                    for (int m = 0; m < MB; ++m) wt[ew * MB + m] = E[m];
                }
                named_sync(kNamedEpi, 128);
                float C[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) C[m] = Sin[m];
#pragma unroll
                for (int ww = 0; ww < 4; ++ww) {
                    if (ww == ew) {
#pragma unroll
                        for (int m = 0; m < MB; ++m) S[m] = C[m];
                    }
                    float w2[MB];
                    matvec_f32<MB>(sP + 5 * MB * MB, C, w2);
#pragma unroll
                    for (int m = 0; m < MB; ++m) C[m] = w2[m] + wt[ww * MB + m];
                }
#pragma unroll
                for (int m = 0; m < MB; ++m) Sin[m] = C[m];
                float v[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) v[m] = S[m];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if ((lane >> k) & 1) {
                        float w2[MB];
                        matvec_f32<MB>(sP + k * MB * MB, v, w2);
#pragma unroll
                        for (int m = 0; m < MB; ++m) v[m] = w2[m];
                    }
                }
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    const float wprev = __shfl_up_sync(0xffffffffu, E[m], 1);
                    S[m] = v[m] + (lane > 0 ? wprev : 0.f);
                }
                if (et == 0) bulk_wait_read0();   // the y buffer's previous store has read it
                named_sync(kNamedEpi, 128);       // wt reusable, y buffer writable
            } else {
                float *xbuf = reinterpret_cast<float *>(lo);
                float *sbuf = reinterpret_cast<float *>(lo + 16384);
                if (et == 0) bulk_wait_read0();   // the y buffer's previous store has read it
                named_sync(kNamedEpi, 128);
#pragma unroll
                for (int m = 0; m < MB; ++m) xbuf[et * MB + m] = E[m];
                named_sync(kNamedEpi, 128);
                if constexpr (Tab::kBlockScan)   // scratch in the y buffer's free parts
                    pipe::dw_scan_group_blocked<MB>(sAt, st, xbuf, sbuf, nch, false, et,
                                                    [] { named_sync(kNamedEpi, 128); },
                                                    reinterpret_cast<float2 *>(lo + 8192),
                                                    reinterpret_cast<float2 *>(lo + 24576));
                else
                    pipe::dw_scan_group<MB>(sAt, st, xbuf, sbuf, nch, false, et,
                                            [] { named_sync(kNamedEpi, 128); });
                if ((nch & 1) && et < MB) st[et] = st[MB + et];   // outgoing state to st[0]
                named_sync(kNamedEpi, 128);
#pragma unroll
                for (int m = 0; m < MB; ++m) S[m] = et < nch ? sbuf[et * MB + m] : 0.f;
                named_sync(kNamedEpi, 128);
            }
            if (saved && et < nch) {
                float *dst = saved + (size_t)(pv.chunk0 + et) * bt.Mstride;
#pragma unroll
                for (int m = 0; m < MB; ++m)
                    if (m < pv.M) dst[m] = S[m];
            }
            // y = D + O_L S, staged in the operand layout (row = chunk, two K blocks)
#pragma unroll 1
            for (int cb = 0; cb < kL / 16; ++cb) {
                float v[16];
                tmem_ld16(taddr + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float *ol = sOL + (cb * 16 + q) * MB;
                    float acc = v[q];
#pragma unroll
                    for (int m = 0; m < MB; ++m) acc = fmaf(ol[m], S[m], acc);
                    v[q] = acc;
                }
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int j16 = cb * 4 + p;
                    *reinterpret_cast<float4 *>(lo + op_piece(et, j16)) =
                        make_float4(v[4 * p], v[4 * p + 1], v[4 * p + 2], v[4 * p + 3]);
                }
            }
            tc_fence_before();
            fence_proxy_async_smem();
            named_sync(kNamedEpi, 128);
            const bool tma_store = use_tma && pv.tlen == kTileSamples;
            if (et == 0) {
                mbar_arrive(&tmem_free[s]);
                if (tma_store) {
                    // asynchronous: the next tile waits for the read of this buffer
                    const int row = (int)(pv.tstart / kL);
                    tma_store_3d(&tmy, 0, 0, row, sbase + PS::YS);
                    tma_store_3d(&tmy, 0, 1, row, sbase + PS::YS + kKBlock);
                    bulk_commit();
                }
                if (pv.last) mbar_arrive(&tab_free[pv.tab]);
            }
            if (!tma_store) {
                const bool al = y_al && ((pv.tstart & 3) == 0);
#pragma unroll 4
                for (int q = 0; q < 16; ++q) {
                    const int id = et + 128 * q;
                    const int r = id >> 4, j16 = id & 15;
                    const float4 v = *reinterpret_cast<const float4 *>(lo + op_piece(r, j16));
                    const int sidx = r * kL + j16 * 4;
                    const int nv = min(max(pv.tlen - sidx, 0), 4);
                    float *gp = y + pv.tstart + sidx;
                    if (nv == 4 && al) {
                        *reinterpret_cast<float4 *>(gp) = v;
                    } else {
                        if (nv > 0) gp[0] = v.x;
                        if (nv > 1) gp[1] = v.y;
                        if (nv > 2) gp[2] = v.z;
                        if (nv > 3) gp[3] = v.w;
                    }
                }
            }
        }
        if (et == 0) bulk_wait0();   // every TMA store complete before the CTA exits
    }
    // ---- exit (the MMA warp drained its tensor-core work above) ----
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int MB, bool F64>
cudaError_t launch_fwd_ws(const float *x, const float *zi, float *y, float *saved, const char *tabs,
                          unsigned long long *counter,
                          const Batch &bt, int three, int num_sms, cudaStream_t st) {
    constexpr int NST = fwd_stages<MB, F64>();
    using SM = WsSmem<MB, F64, NST>;
    static_assert(SM::ALLOC <= kSmemMax, "shared memory budget");
    auto kern = chunk_fwd_ws_kernel<MB, F64, NST>;
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::ALLOC);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const int64_t grid = bt.B < num_sms ? bt.B : num_sms;
    const int x_al = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    const int y_al = (reinterpret_cast<uintptr_t>(y) & 15) == 0;
    // TMA needs chunk-aligned channel starts (fixed shape, T a multiple of L)
    CUtensorMap tmx, tmy;
    std::memset(&tmx, 0, sizeof(tmx));
    std::memset(&tmy, 0, sizeof(tmy));
    int use_tma = 0;
    if (!bt.offsets && bt.T % kL == 0 && make_chunk_tmap(&tmx, x, bt.total) &&
        make_chunk_tmap(&tmy, y, bt.total))
        use_tma = 1;
    kern<<<(unsigned)grid, kFwdThreads, SM::ALLOC, st>>>(x, zi, y, saved, tabs, counter, bt, three, x_al,
                                                       y_al, use_tma, tmx, tmy); note_launch();
    return cudaGetLastError();
}

}  // namespace

template <int MB>
cudaError_t chunk_fwd_mb(const float *x, const float *zi, float *y, float *saved, const char *tabs,
                         unsigned long long *counter,
                         const Batch &bt, bool fp64_scan, int three, int num_sms, cudaStream_t st) {
    // pipelined kernel wherever its double-buffered layout fits the shared memory
    if constexpr (WsSmem<MB, true, fwd_stages<MB, true>()>::ALLOC <= kSmemMax)
        if (fp64_scan) return launch_fwd_ws<MB, true>(x, zi, y, saved, tabs, counter, bt, three, num_sms, st);
    if constexpr (MB <= kMaxF32ScanBucket &&
                  WsSmem<MB, false, fwd_stages<MB, false>()>::ALLOC <= kSmemMax)
        if (!fp64_scan) return launch_fwd_ws<MB, false>(x, zi, y, saved, tabs, counter, bt, three, num_sms, st);
    if (fp64_scan) return launch_fwd_t<MB, true>(x, zi, y, saved, tabs, counter, bt, three, num_sms, st);
    if constexpr (MB <= kMaxF32ScanBucket)
        return launch_fwd_t<MB, false>(x, zi, y, saved, tabs, counter, bt, three, num_sms, st);
    return cudaErrorNotSupported;
}

template cudaError_t chunk_fwd_mb<DFILT_MB>(const float *, const float *, float *, float *,
                                            const char *, unsigned long long *, const Batch &, bool,
                                            int, int, cudaStream_t);

}  // namespace dfilt
