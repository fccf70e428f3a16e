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
#include "chunk.cuh"

#ifndef DFILT_MB
#error "compile once per state bucket with -DDFILT_MB=<2|4|8|16|32|64>"
#endif

namespace dfilt {

namespace {

constexpr int kThreads = 128;
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
    // misc block: mbarrier (8) | tmem base (4) | channel (8) | flag (4) | drill mbarrier (8) | S_in (MB doubles)
    static constexpr uint32_t BYTES = MISC + 48 + MB * 8;
    static constexpr uint32_t ALLOC = BYTES + 1024;   // slack for 1024-byte alignment
};

// Load samples [start, start+n) of src into the swizzled A tile at `dst` (2 K blocks),
// zero-filling past n.  Thread t handles the 16-byte pieces t, t+128, ...
__device__ __forceinline__ void load_tile(uint32_t dst, const float *src, int64_t start, int n,
                                          bool al16) {
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
        const int id = threadIdx.x + kThreads * q;
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
__device__ __forceinline__ void split_tile(char *smem, uint32_t a_off, uint32_t lo_off, bool three) {
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
        const int id = threadIdx.x + kThreads * q;
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
__device__ __forceinline__ void store_tile(float *dst, int64_t start, int n, const char *stag,
                                           bool al16) {
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
        const int id = threadIdx.x + kThreads * q;
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
                     float *__restrict__ y, float *__restrict__ saved, const char *__restrict__ ws,
                     unsigned long long *__restrict__ counter, Batch bt, int three, int x_al,
                     int y_al) {
    using Tab = ChunkTab<MB>;
    using SM = FwdSmem<MB, F64>;
    constexpr int NM = SM::NM;
    extern __shared__ char smem_raw[];
    char *smem = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + SM::MISC);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM::MISC + 8);
    int64_t *ch_slot = reinterpret_cast<int64_t *>(smem + SM::MISC + 16);
    int *flag_slot = reinterpret_cast<int *>(smem + SM::MISC + 24);
    double *sin_buf = reinterpret_cast<double *>(smem + SM::MISC + 48);
    float *sOL = reinterpret_cast<float *>(smem + SM::OL);
    const float *sP = reinterpret_cast<const float *>(smem + SM::SCAN);
    const double *sAt = reinterpret_cast<const double *>(smem + SM::SCAN);

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
    const size_t rec = Tab::fwd_rec(F64);
    constexpr uint32_t idesc = idesc_tf32_m128(NM);

    while (alive) {
        if (tid == 0) *ch_slot = (int64_t)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t ch = *ch_slot;
        if (ch >= bt.B) break;
        const Channel c = channel_of(bt, ch);
        const char *R = ws + kWsHeader + (size_t)ch * rec;
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

        // per-thread carried state for the FP32 scan; warp 0 carries the FP64 one
        float Sin[MB];
        double S64a = 0.0, S64b = 0.0;
#pragma unroll
        for (int m = 0; m < MB; ++m) Sin[m] = (float)sin_buf[m];
        if (F64 && warp == 0) {
            S64a = lane < MB ? sin_buf[lane] : 0.0;
            S64b = lane + 32 < MB ? sin_buf[lane + 32] : 0.0;
        }
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
                // serial FP64 scan by warp 0: S_{c+1} = Abar S_c + E_c, state carried in FP64
                float *sbuf = reinterpret_cast<float *>(smem + SM::AHI);
#pragma unroll
                for (int m = 0; m < MB; ++m) xbuf[tid * MB + m] = E[m];
                __syncthreads();
                if (warp == 0) {
                    for (int cc = 0; cc < nch; ++cc) {
                        if (lane < MB) sbuf[cc * MB + lane] = (float)S64a;
                        if (lane + 32 < MB) sbuf[cc * MB + lane + 32] = (float)S64b;
                        double acc_a = lane < MB ? (double)xbuf[cc * MB + lane] : 0.0;
                        double acc_b = lane + 32 < MB ? (double)xbuf[cc * MB + lane + 32] : 0.0;
#pragma unroll 8
                        for (int j = 0; j < MB; ++j) {
                            const double sj = __shfl_sync(0xffffffffu, j < 32 ? S64a : S64b, j & 31);
                            if (lane < MB) acc_a = fma(sAt[j * MB + lane], sj, acc_a);
                            if (lane + 32 < MB) acc_b = fma(sAt[j * MB + lane + 32], sj, acc_b);
                        }
                        S64a = acc_a;
                        S64b = acc_b;
                    }
                }
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
cudaError_t launch_fwd_t(const float *x, const float *zi, float *y, float *saved, const char *ws,
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
    auto *counter = reinterpret_cast<unsigned long long *>(const_cast<char *>(ws));
    kern<<<(unsigned)grid, kThreads, SM::ALLOC, st>>>(x, zi, y, saved, ws, counter, bt, three, x_al, y_al);
    return cudaGetLastError();
}

}  // namespace

template <int MB>
cudaError_t chunk_fwd_mb(const float *x, const float *zi, float *y, float *saved, const char *ws,
                         const Batch &bt, bool fp64_scan, int three, int num_sms, cudaStream_t st) {
    if (fp64_scan) return launch_fwd_t<MB, true>(x, zi, y, saved, ws, bt, three, num_sms, st);
    if constexpr (MB <= kMaxF32ScanBucket)
        return launch_fwd_t<MB, false>(x, zi, y, saved, ws, bt, three, num_sms, st);
    return cudaErrorNotSupported;
}

template cudaError_t chunk_fwd_mb<DFILT_MB>(const float *, const float *, float *, float *,
                                            const char *, const Batch &, bool, int, int,
                                            cudaStream_t);

}  // namespace dfilt
