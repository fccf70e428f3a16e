// Chunked backward (closed-form adjoint of Sec. 3.1) on the tensor cores (sm_103a).
//
// The adjoint u[n] = gy[n] - sum_k a_k u[n+k] (u = 0 past the end, App. A) and
// grad_x = B applied anti-causally to u are the forward machinery run backwards in
// time.  A CTA owns whole channels and walks their tiles from the last to the first.
// Per tile:
//   1. cp.async gy (swizzled K-major A operand, split into TF32 hi/lo) and x (and y
//      when it is given) into shared memory;
//   2. tcgen05.mma: D[128 x 128] = G [T_g^a | T_h^a]^T -- columns 0..63 of row c are
//      chunk c's zero-state grad_x, columns 64..127 its zero-state adjoint u;
//   3. reverse chunk scan of the adjoint state S'_c = u[(c+1)L .. (c+1)L+MB)
//      (S'_{c-1} = Abar' S'_c + u_zs,c[0:MB]), FP32 Hillis-Steele or serial double-word;
//   4. fused epilogue per chunk: u = u_zs + O^u S', grad_x = gx_zs + O^gx S' (stored),
//      y recomputed from the forward's saved chunk state (or read), and the lag
//      correlations grad_b[k] += sum u[n+k] x[n], grad_a[k] -= sum u[n+1+k] y[n]
//      reduced warp-wise into per-CTA FP64 accumulators; grad_zi = u[0:M].
#include <cstring>

#include "chunk_pipe.cuh"

#ifndef DFILT_MB
#error "compile once per state bucket with -DDFILT_MB=<2|4|8|16|32|64>"
#endif

namespace dfilt {

namespace {

constexpr int kThreads = 128;
constexpr uint32_t kTileBytes = kChunks * kL * 4;   // 32 KB
constexpr uint32_t kKBlock = kChunks * 128;

template <int MB, bool F64, bool READ_Y>
struct BwdSmem {
    using Tab = ChunkTab<MB>;
    static constexpr int NM = Tab::NBWD;
    // For MB == L with the serial scan, O^u is read from its transition (Abar' = O^u).
    static constexpr bool OU_FROM_AT = F64 && MB == kL;
    static constexpr uint32_t AHI = 0;
    static constexpr uint32_t ALO = AHI + kTileBytes;
    static constexpr uint32_t BHI = ALO + kTileBytes;
    static constexpr uint32_t BLO = BHI + NM * 256;
    static constexpr uint32_t XS = BLO + NM * 256;
    static constexpr uint32_t YS = XS + kTileBytes;
    static constexpr uint32_t OU = YS + (READ_Y ? kTileBytes : 0);
    static constexpr uint32_t OGX = OU + (OU_FROM_AT ? 0 : kL * MB * 4);
    static constexpr uint32_t SCAN = OGX + kL * MB * 4;
    static constexpr uint32_t COEF = (SCAN + (uint32_t)Tab::scan_bytes(F64) + 15) / 16 * 16;
    static constexpr uint32_t ACC = (COEF + 2 * (MB + 1) * 4 + 15) / 16 * 16;   // 4 x (2MB+1) doubles
    static constexpr uint32_t MISC = ACC + 4 * (2 * MB + 1) * 8;
    static constexpr uint32_t ST = MISC + 48;                 // serial-scan state [2][MB] double words
    static constexpr uint32_t BYTES = ST + 2 * MB * 8;
    static constexpr uint32_t ALLOC = BYTES + 1024;
};

__device__ __forceinline__ void load_tile_sw(uint32_t dst, const float *src, int64_t start, int n,
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
}

// Row-staged tile: row c = chunk c (256 bytes), 16-byte piece j at ((j ^ (c & 15)) << 4).
__device__ __forceinline__ void load_tile_rows(uint32_t dst, const float *src, int64_t start, int n,
                                               bool al16) {
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
        const int id = threadIdx.x + kThreads * q;
        const int r = id >> 4, j = id & 15;
        const uint32_t d = dst + r * 256 + ((j ^ (r & 15)) << 4);
        const int s = r * kL + j * 4;
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
}

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

__device__ __forceinline__ float4 row_piece(const char *buf, int r, int j) {
    return *reinterpret_cast<const float4 *>(buf + r * 256 + ((j ^ (r & 15)) << 4));
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

template <int MB, bool F64, bool READ_Y>
__global__ void __launch_bounds__(kThreads, 1)
    chunk_bwd_kernel(const float *__restrict__ gy, const float *__restrict__ x,
                     const float *__restrict__ y, const float *__restrict__ b,
                     const float *__restrict__ a, const float *__restrict__ saved,
                     float *__restrict__ gx, float *__restrict__ gb, float *__restrict__ ga,
                     float *__restrict__ gzi, const char *__restrict__ tabs,
                     unsigned long long *__restrict__ counter, Batch bt, int three, int al_mask) {
    using Tab = ChunkTab<MB>;
    using SM = BwdSmem<MB, F64, READ_Y>;
    constexpr int NM = SM::NM;
    constexpr int NACC = 2 * MB + 1;
    extern __shared__ char smem_raw[];
    char *smem = smem_align1024(smem_raw);
    const uint32_t sbase = smem_u32(smem);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + SM::MISC);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM::MISC + 8);
    int64_t *ch_slot = reinterpret_cast<int64_t *>(smem + SM::MISC + 16);
    int *flag_slot = reinterpret_cast<int *>(smem + SM::MISC + 24);
    float *sOU = reinterpret_cast<float *>(smem + SM::OU);
    float *sOGX = reinterpret_cast<float *>(smem + SM::OGX);
    const float *sP = reinterpret_cast<const float *>(smem + SM::SCAN);
    const float2 *sAt = reinterpret_cast<const float2 *>(smem + SM::SCAN);
    float *sa = reinterpret_cast<float *>(smem + SM::COEF);
    float *sb = sa + (MB + 1);
    double *sacc = reinterpret_cast<double *>(smem + SM::ACC);

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
    const size_t rec = bt.bwd_stride ? (size_t)bt.bwd_stride : Tab::bwd_rec(F64);
    constexpr uint32_t idesc = idesc_tf32_m128(NM);
    const bool gy_al = al_mask & 1, x_al = al_mask & 2, y_al = al_mask & 4, gx_al = al_mask & 8;

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
        {
            const float *g = reinterpret_cast<const float *>(R + Tab::B_G);
            const float *h = reinterpret_cast<const float *>(R + Tab::B_H);
            for (int idx = tid; idx < NM * kL; idx += kThreads) {
                const int i = idx / kL, k = idx % kL;
                // row i < L: grad_x output i, T_g^a[i][k] = g[k-i]; row L+i: u output i
                const int ii = i < kL ? i : i - kL;
                const float *imp = i < kL ? g : h;
                const float v = k >= ii ? imp[k - ii] : 0.f;
                float hv, lv;
                split_tf32(v, hv, lv);
                const uint32_t o = (k >> 5) * (NM * 128) + sw128_off(i, k & 31);
                *reinterpret_cast<float *>(smem + SM::BHI + o) = hv;
                *reinterpret_cast<float *>(smem + SM::BLO + o) = lv;
            }
            if constexpr (!SM::OU_FROM_AT) {
                const float *Ou = reinterpret_cast<const float *>(R + Tab::B_OU);
                for (int idx = tid; idx < kL * MB; idx += kThreads) sOU[idx] = Ou[idx];
            }
            const float *Ogx = reinterpret_cast<const float *>(R + Tab::B_OGX);
            for (int idx = tid; idx < kL * MB; idx += kThreads) sOGX[idx] = Ogx[idx];
            const float4 *src = reinterpret_cast<const float4 *>(R + Tab::B_SCAN);
            float4 *dst = reinterpret_cast<float4 *>(smem + SM::SCAN);
            for (int idx = tid; idx < (int)(Tab::scan_bytes(F64) / 16); idx += kThreads) dst[idx] = src[idx];
            if (tid < MB) sa[tid] = tid < c.M ? a[ch * bt.Mstride + tid] : 0.f;
            if (tid <= MB) sb[tid] = tid <= c.N ? b[ch * bt.Nstride + tid] : 0.f;
            for (int idx = tid; idx < 4 * NACC; idx += kThreads) sacc[idx] = 0.0;
        }
        fence_proxy_async_smem();
        __syncthreads();

        float Sin[MB];   // adjoint state entering the current tile from the right
        float2 *st = reinterpret_cast<float2 *>(smem + SM::ST);   // serial-scan state
#pragma unroll
        for (int m = 0; m < MB; ++m) Sin[m] = 0.f;
        if (F64 && tid < MB) st[tid] = make_float2(0.f, 0.f);
        const int64_t ntiles = (c.len + kTileSamples - 1) / kTileSamples;
        const int64_t chunk_base = c.off / kL + ch;

        for (int64_t t = ntiles - 1; t >= 0; --t) {
            const int64_t tstart = c.off + t * kTileSamples;
            const int tlen = (int)(c.len - t * kTileSamples < kTileSamples ? c.len - t * kTileSamples : kTileSamples);
            const int nch = (tlen + kL - 1) / kL;
            const bool a4 = (tstart & 3) == 0;
            load_tile_sw(sbase + SM::AHI, gy, tstart, tlen, gy_al && a4);
            load_tile_rows(sbase + SM::XS, x, tstart, tlen, x_al && a4);
            if constexpr (READ_Y) load_tile_rows(sbase + SM::YS, y, tstart, tlen, y_al && a4);
            cp_async_commit();
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

            // ---- E'_c = u_zs[0:MB] (TMEM columns L .. L+MB) ----
            float E[MB];
#pragma unroll
            for (int cb = 0; cb < (MB + 15) / 16; ++cb) {
                float v[16];
                tmem_ld16(taddr + kL + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (cb * 16 + i < MB) E[cb * 16 + i] = v[i];
            }
            float S[MB];   // S'_c: adjoint values u[(c+1)L + m]
            float *xbuf = reinterpret_cast<float *>(smem + SM::ALO);
            if constexpr (!F64) {
                // Two-level reverse scan.  (1) warp-local: W'_c = sum_{j=c..32w+31} Abar'^(j-c) E'_j
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int d = 1 << k;
                    float nxt[MB];
#pragma unroll
                    for (int m = 0; m < MB; ++m) nxt[m] = __shfl_down_sync(0xffffffffu, E[m], d);
                    if (lane + d < 32) {
                        float add[MB];
                        matvec_f32<MB>(sP + k * MB * MB, nxt, add);
#pragma unroll
                        for (int m = 0; m < MB; ++m) E[m] += add[m];
                    }
                }
                // (2) carries from the right: C'_3 = S'_in, C'_{w-1} = Abar'^32 C'_w + W'_{32w}
                // (state entering chunk 32w+31 from the right); the last one leaves the tile
                if (lane == 0) {
#pragma unroll
                    for (int m = 0; m < MB; ++m) xbuf[warp * MB + m] = E[m];
                }
                __syncthreads();
                float C[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) C[m] = Sin[m];
                for (int ww = kChunks / 32 - 1; ww >= 0; --ww) {
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
                // (3) state entering chunk c = 32w + l from the right: Abar'^(31-l) C'_w + W'_{c+1}
                float v[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) v[m] = S[m];
                const int e = 31 - lane;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if ((e >> k) & 1) {
                        float w2[MB];
                        matvec_f32<MB>(sP + k * MB * MB, v, w2);
#pragma unroll
                        for (int m = 0; m < MB; ++m) v[m] = w2[m];
                    }
                }
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    const float wnext = __shfl_down_sync(0xffffffffu, E[m], 1);
                    S[m] = v[m] + (lane < 31 ? wnext : 0.f);
                }
                __syncthreads();
            } else {
                float *sbuf = reinterpret_cast<float *>(smem + SM::AHI);
#pragma unroll
                for (int m = 0; m < MB; ++m) xbuf[tid * MB + m] = E[m];
                __syncthreads();
                if constexpr (Tab::kBlockScan)   // scratch in the A_lo tile behind E
                    pipe::dw_scan_group_blocked<MB>(sAt, st, xbuf, sbuf, nch, true, tid,
                                                    [] { __syncthreads(); },
                                                    reinterpret_cast<float2 *>(smem + SM::ALO + 8192),
                                                    reinterpret_cast<float2 *>(smem + SM::ALO + 16384));
                else
                    pipe::dw_scan_group<MB>(sAt, st, xbuf, sbuf, nch, true, tid, [] { __syncthreads(); });
                if ((nch & 1) && tid < MB) st[tid] = st[MB + tid];   // outgoing state to st[0]
                __syncthreads();
#pragma unroll
                for (int m = 0; m < MB; ++m) S[m] = tid < nch ? sbuf[tid * MB + m] : 0.f;
                __syncthreads();
            }

            // ---- y for this chunk: read, or recomputed from the forward's chunk state ----
            float yv[kL];
            if constexpr (READ_Y) {
#pragma unroll
                for (int j = 0; j < kL / 4; ++j) {
                    const float4 p = row_piece(smem + SM::YS, tid, j);
                    yv[4 * j] = p.x; yv[4 * j + 1] = p.y; yv[4 * j + 2] = p.z; yv[4 * j + 3] = p.w;
                }
            } else {
                float s[MB];
                const bool vch = tid < nch;
                const float *src = saved + (size_t)(chunk_base + t * kChunks + tid) * bt.Mstride;
#pragma unroll
                for (int m = 0; m < MB; ++m) s[m] = (vch && m < c.M) ? src[m] : 0.f;
#pragma unroll
                for (int j = 0; j < kL / 4; ++j) {
                    const float4 p = row_piece(smem + SM::XS, tid, j);
                    const float xs4[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float xn = xs4[e];
                        const float yn = fmaf(sb[0], xn, s[0]);
#pragma unroll
                        for (int k = 0; k < MB; ++k)
                            s[k] = fmaf(-sa[k], yn, fmaf(sb[k + 1], xn, k + 1 < MB ? s[k + 1] : 0.f));
                        yv[4 * j + e] = yn;
                    }
                }
            }

            // ---- u and grad_x for this chunk; correlations ----
            float u[kL];
            char *stag = smem + SM::AHI;   // gy tile is no longer needed
            float pb[MB + 1], pa[MB];
#pragma unroll
            for (int k = 0; k <= MB; ++k) pb[k] = 0.f;
#pragma unroll
            for (int k = 0; k < MB; ++k) pa[k] = 0.f;
#pragma unroll
            for (int cb = 0; cb < kL / 16; ++cb) {
                float vu[16], vg[16];
                tmem_ld16(taddr + kL + cb * 16, vu);
                tmem_ld16(taddr + cb * 16, vg);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = cb * 16 + i;
                    float au = vu[i], ag = vg[i];
#pragma unroll
                    for (int m = 0; m < MB; ++m) {
                        const float ou = SM::OU_FROM_AT ? dw_to_float(dw{sAt[m * MB + n].x, sAt[m * MB + n].y})
                                                        : sOU[n * MB + m];
                        au = fmaf(ou, S[m], au);
                        ag = fmaf(sOGX[n * MB + m], S[m], ag);
                    }
                    u[n] = au;
                    vg[i] = ag;
                }
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int j = cb * 4 + p;
                    *reinterpret_cast<float4 *>(stag + tid * 256 + ((j ^ (tid & 15)) << 4)) =
                        make_float4(vg[4 * p], vg[4 * p + 1], vg[4 * p + 2], vg[4 * p + 3]);
                }
            }
            // ext[n] = u[n] for n < L, S'[n - L] above
#define DFILT_EXT(n) ((n) < kL ? u[(n)] : S[(n) - kL])
#pragma unroll
            for (int j = 0; j < kL / 4; ++j) {
                const float4 p = row_piece(smem + SM::XS, tid, j);
                const float xs4[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int n = 4 * j + e;
#pragma unroll
                    for (int k = 0; k <= MB; ++k) pb[k] = fmaf(DFILT_EXT(n + k), xs4[e], pb[k]);
#pragma unroll
                    for (int k = 0; k < MB; ++k) pa[k] = fmaf(DFILT_EXT(n + 1 + k), yv[n], pa[k]);
                }
            }
#undef DFILT_EXT
            if (gzi && t == 0 && tid == 0) {
#pragma unroll
                for (int m = 0; m < MB; ++m)
                    if (m < c.M) gzi[ch * bt.Mstride + m] = (m < c.len) ? u[m] : 0.f;
            }
            // warp reduction of the correlations, then into the CTA's FP64 accumulators
#pragma unroll
            for (int k = 0; k < NACC; ++k) {
                float v = k <= MB ? pb[k] : pa[k - MB - 1];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) sacc[warp * NACC + k] += (double)v;
            }
            tc_fence_before();
            __syncthreads();
            if (gx) store_tile(gx, tstart, tlen, stag, gx_al && a4);
            __syncthreads();
        }
        if (!alive) break;
        // ---- channel done: coefficient gradients ----
        for (int k = tid; k < NACC; k += kThreads) {
            const double v = sacc[k] + sacc[NACC + k] + sacc[2 * NACC + k] + sacc[3 * NACC + k];
            if (k <= MB) {
                if (gb && k <= c.N) gb[ch * bt.Nstride + k] = (float)v;
            } else {
                const int m = k - MB - 1;
                if (ga && m < c.M) ga[ch * bt.Mstride + m] = (float)(-v);
            }
        }
        if (gzi && c.len == 0 && tid < c.M) gzi[ch * bt.Mstride + tid] = 0.f;
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 128);
    }
}

template <int MB, bool F64, bool READ_Y>
cudaError_t launch_bwd_t(const float *gy, const float *x, const float *y, const float *b,
                         const float *a, const float *saved, float *gx, float *gb, float *ga,
                         float *gzi, const char *tabs, unsigned long long *counter, const Batch &bt, int three, int num_sms,
                         cudaStream_t st) {
    using SM = BwdSmem<MB, F64, READ_Y>;
    static_assert(SM::ALLOC <= 232448, "shared memory budget");
    auto kern = chunk_bwd_kernel<MB, F64, READ_Y>;
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
        occ[dev] = o < 1 ? 1 : (o > 2 ? 2 : o);
    }
    const int64_t slots = (int64_t)num_sms * occ[dev];
    const int64_t grid = bt.B < slots ? bt.B : slots;
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const int mask = (al(gy) ? 1 : 0) | (al(x) ? 2 : 0) | ((y && al(y)) ? 4 : 0) | ((gx && al(gx)) ? 8 : 0);
    kern<<<(unsigned)grid, kThreads, SM::ALLOC, st>>>(gy, x, y, b, a, saved, gx, gb, ga, gzi, tabs,
                                                      counter, bt, three, mask); note_launch();
    return cudaGetLastError();
}


// ===========================================================================
// Warp-specialised backward (state buckets whose layout fits), the forward's
// pipeline structure run on reversed tiles, with two epilogue warpgroups:
//   warps 0-3   converters: work (tiles of a channel from last to first), tables (the
//               B operand T_h^a, O^u, scan block, coefficients, built from the channel's
//               record staged by a bulk copy; double-buffered by channel parity); gy
//               tiles two ahead into two stages (TMA or cp.async); warp w writes the
//               TF32 operand of rows 32w .. 32w+31 (the raw words as hi, x - trunc(x)
//               as lo) into TMEM operand slot i&1 -> full[s], after which the stage is
//               free
//   warp 12     MMA: D[128 x 64] = G T_h^a^T (zero-state adjoint u per chunk; A from
//               TMEM, the B operand from shared memory) into TMEM accumulator i&3
//   warps 4-7   epilogue group 0 (even tiles), warps 8-11 group 1 (odd tiles): reverse
//               chunk scan of S'_c = u[(c+1)L ..] (each group loads its tile's x into its
//               own buffer, issued before it waits for the tile's accumulator; the state
//               entering from the right is the other group's carry), u = D + O^u S',
//               then streamed over the chunk row: y recomputed
//               from the forward's saved chunk state and the x tile, lag correlations,
//               grad_x = sum_k b_k u[n+k] written over the x tile and stored from there
//               (TMA for full tiles); lag sums added per channel in shared FP64, finished
//               by the group that completes the channel's last tile
// ===========================================================================

// 13 warps: converters 0-3 (one per TMEM lane quarter), epilogue groups 4-7 and 8-11,
// MMA issuer 12
constexpr int kBwThreads = 416;
constexpr int kBwConv = 128;     // converter threads
constexpr int kBwMmaWarp = 12;
constexpr int kBwNS = 2;   // gy stages (a stage is free once converted; loads run two ahead)
constexpr int kBwNX = 2;   // x / grad_x buffers (one per epilogue group)

template <int MB, bool F64>
struct BwSmem {
    using Tab = ChunkTab<MB>;
    static constexpr int NM = kL;                                    // MMA N: T_h^a rows
    static constexpr int NACC = 2 * MB + 1;
    static constexpr uint32_t GS0 = 0;                               // gy stages (hi)
    static constexpr uint32_t XB0 = kBwNS * pipe::kTileBytes;        // x / grad_x buffers
    static constexpr uint32_t TB = XB0 + kBwNX * pipe::kTileBytes;   // 2 slots: B operand hi | lo
    static constexpr uint32_t T_BHI = 0;                             // within a B slot
    static constexpr uint32_t T_BLO = NM * 256;
    static constexpr uint32_t BSLOT = 2 * NM * 256;
    static constexpr uint32_t SMALL0 = TB + 2 * BSLOT;               // 2 slots: O^u | scan | coef
    static constexpr uint32_t S_OU = 0;
    static constexpr uint32_t S_SCAN = kL * MB * 4;
    static constexpr uint32_t S_COEF = (S_SCAN + (uint32_t)Tab::scan_bytes(F64) + 15) / 16 * 16;
    static constexpr uint32_t SSLOT = (S_COEF + (2 * MB + 1) * 4 + 15) / 16 * 16;
    // staging of a channel's record (bulk copy): h | O^u, then scan block | coefficients
    static constexpr uint32_t G_PART0 = (uint32_t)(Tab::B_OGX - Tab::B_H);
    static constexpr uint32_t G_PART1 = (uint32_t)(Tab::b_coef(F64) + Tab::COEF_BYTES - Tab::B_SCAN);
    static constexpr uint32_t G_COEF = G_PART0 + (uint32_t)(Tab::b_coef(F64) - Tab::B_SCAN);
    static constexpr uint32_t STG = (SMALL0 + 2 * SSLOT + 127) / 128 * 128;
    // FP64 reverse scan scratch per group (E' and S' per chunk)
    static constexpr uint32_t SCR = (STG + G_PART0 + G_PART1 + 15) / 16 * 16;
    static constexpr uint32_t SCR_G = F64 ? 2 * kChunks * MB * 4 + 2 * MB * 8 : 0;   // + scan state
    // lag sums per [table slot][group][warp][NACC] doubles: one writer per slot, so every
    // partial sum runs in a fixed order
    static constexpr uint32_t ACC = (SCR + 2 * SCR_G + 7) / 8 * 8;
    static constexpr uint32_t CNT = ACC + 16 * NACC * 8;             // tiles done [2 slots]
    static constexpr uint32_t CARRY = CNT + 16;                      // [2][MB] floats
    static constexpr uint32_t CARRY64 = (CARRY + 2 * MB * 4 + 7) / 8 * 8;   // [2][MB] doubles
    static constexpr uint32_t MISC = (CARRY64 + 2 * MB * 8 + 15) / 16 * 16;
    static constexpr int NBAR = 26;
    static constexpr uint32_t M_BAR = MISC;
    static constexpr uint32_t M_TMEM = MISC + NBAR * 8;
    static constexpr uint32_t M_ABORT = M_TMEM + 4;
    static constexpr uint32_t M_OK = M_TMEM + 16;    // 12 flags: converters 4, groups 4 + 4
    static constexpr uint32_t M_WT = M_OK + 48;      // [2 groups][4 warps][MB] floats
    static constexpr uint32_t M_RING = (M_WT + 2 * 4 * MB * 4 + 15) / 16 * 16;
    static constexpr uint32_t BYTES = M_RING + 8 * 48;
    static constexpr uint32_t ALLOC = BYTES + 1024;
};

template <int MB, bool F64>
__global__ void __launch_bounds__(kBwThreads, 1)
    chunk_bwd_ws_kernel(const float *__restrict__ gy, const float *__restrict__ x,
                        const float *__restrict__ bco, const float *__restrict__ aco,
                        const float *__restrict__ saved,
                        float *__restrict__ gx, float *__restrict__ gb, float *__restrict__ ga,
                        float *__restrict__ gzi, const char *__restrict__ tabs,
                        unsigned long long *__restrict__ counter, Batch bt, int three, int al_mask,
                        int tma_mask, const __grid_constant__ CUtensorMap tmg,
                        const __grid_constant__ CUtensorMap tmx,
                        const __grid_constant__ CUtensorMap tmgx) {
    using namespace pipe;
    using Tab = ChunkTab<MB>;
    using SM = BwSmem<MB, F64>;
    constexpr int NM = SM::NM;
    constexpr int NACC = SM::NACC;
    static_assert(NACC <= 32, "one lag product per lane");
    extern __shared__ char smem_raw[];
    char *smem = smem_align1024(smem_raw);
    const uint32_t sbase = smem_u32(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SM::M_BAR);
    uint64_t *full = bars + 0, *load_bar = bars + 6, *mma_done = bars + 9,
             *tmem_free = bars + 13, *x_bar = bars + 17, *tab_free = bars + 19, *carry_bar = bars + 21,
             *dead = bars + 23, *drain = bars + 24, *stg_bar = bars + 25;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM::M_TMEM);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + SM::M_ABORT);
    // decision flags written by one thread and read by its role after a named barrier;
    // each decision point has its own word, so that a late reader never sees the value
    // of a later point (the roles must leave their loops at the same point)
    volatile int *conv_ok = reinterpret_cast<volatile int *>(smem + SM::M_OK);
    double *acc_ch = reinterpret_cast<double *>(smem + SM::ACC);
    unsigned *tiles_done = reinterpret_cast<unsigned *>(smem + SM::CNT);
    float *carry = reinterpret_cast<float *>(smem + SM::CARRY);
    float2 *carry64 = reinterpret_cast<float2 *>(smem + SM::CARRY64);   // double-word carries
    TileDesc *ring = reinterpret_cast<TileDesc *>(smem + SM::M_RING);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool gy_al = al_mask & 1, x_al = al_mask & 2, gx_al = al_mask & 8;
    const bool tma_gy = tma_mask & 1, tma_x = tma_mask & 2, tma_gx = tma_mask & 4;

    if (warp == 0) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < SM::NBAR; ++i) {
            uint32_t cnt = 1;
            if (i >= 9 && i < 13) cnt = 2;                                    // mma_done: commit + arrive
            if (i >= 17 && i < 19 && !tma_x) cnt = 128;                       // x_bar: a group's cp.async arrivals
            mbar_init(&bars[i], cnt);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int i = tid; i < 16 * NACC; i += kBwThreads) acc_ch[i] = 0.0;
    if (tid < 2) tiles_done[tid] = 0u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const size_t rec = bt.bwd_stride ? (size_t)bt.bwd_stride : Tab::bwd_rec(F64);
    auto stage_hi = [&](int s) { return (uint32_t)(SM::GS0 + s * kTileBytes); };
    auto xbuf = [&](int j) { return (uint32_t)(SM::XB0 + j * kTileBytes); };
    auto sslot = [&](int p) { return (uint32_t)(SM::SMALL0 + p * SM::SSLOT); };
    // TMEM: accumulator buffer j (tile i uses j = i & 3) at columns 64 j; operand slot p
    // (tile i uses p = i & 1): A_hi at 256 + 128 p, A_lo at 256 + 128 p + 64
    auto ahi_col = [&](int p) { return (uint32_t)(256 + 128 * p); };
    auto alo_col = [&](int p) { return (uint32_t)(256 + 128 * p + 64); };
    auto wait1 = [&](uint64_t *bar, uint32_t parity) -> bool {
        return wait_or_abort(bar, parity, bt.wait_limit, abort_flag, bt.status);
    };
    // The TF32 operand of the rows of TMEM lane quarter `q` of stage s's gy tile into TMEM
    // operand slot p (one warp, thread = chunk row): the raw word as A_hi (the tensor
    // cores truncate a TF32 operand to its upper 19 bits) and x - trunc(x) as A_lo;
    // samples past the tile's end are zero
    auto a_to_tmem = [&](int q, int n, int s, int p) {
        const int r = 32 * q + lane;
        const char *hi = smem + stage_hi(s);
        const int nv = n - r * kL;
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
        if (__all_sync(0xffffffffu, nv >= kL)) rows(BoolC<true>{});
        else rows(BoolC<false>{});
        tmem_wait_st();
        tc_fence_before();
    };

    if (warp < 4) {
        // ============================ converters ============================
        const int ct = tid;
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
                if (cur_nt == 0) {
                    // an empty channel still owes zero coefficient gradients
                    for (int k = 0; k <= cc.N; ++k)
                        if (gb) gb[c * bt.Nstride + k] = 0.f;
                    for (int k = 0; k < cc.M; ++k) {
                        if (ga) ga[c * bt.Mstride + k] = 0.f;
                        if (gzi) gzi[c * bt.Mstride + k] = 0.f;
                    }
                    continue;
                }
                ++ch_seq;
            }
            const int64_t t = cur_nt - 1 - cur_t;   // reversed time
            d.ch = cur_ch;
            d.tstart = cur_off + t * kTileSamples;
            d.tlen = (int)(cur_len - t * kTileSamples < kTileSamples ? cur_len - t * kTileSamples
                                                                     : kTileSamples);
            d.chunk0 = cur_off / kL + cur_ch + t * kChunks;
            d.tab = ch_seq & 1;
            d.seq = ch_seq;
            d.first = cur_t == 0;
            d.M = cur_M;
            ++cur_t;
            d.last = cur_t == cur_nt;
        };
        // a channel's record (h, O^u, scan block, coefficients) into the staging area:
        // two bulk copies on stg_bar, issued by thread 0 ahead of the table build
        bool stg_pending = false;   // thread 0: a record copy not yet waited for
        auto prefetch_record = [&](const TileDesc &d) {
            const char *R = tabs + (size_t)d.ch * rec;
            stg_pending = true;
            fence_proxy_async_smem();   // the previous build's reads of the area come first
            mbar_arrive_expect_tx(stg_bar, SM::G_PART0 + SM::G_PART1);
            bulk_load(sbase + SM::STG, R + Tab::B_H, SM::G_PART0, stg_bar);
            bulk_load(sbase + SM::STG + SM::G_PART0, R + Tab::B_SCAN, SM::G_PART1, stg_bar);
        };
        // the channel-parity slots of the B operand and of the small tables, from the
        // staged record
        auto build_tables = [&](const TileDesc &d) {
            char *T = smem + sslot(d.tab);
            const char *G = smem + SM::STG;
            const float *hs = reinterpret_cast<const float *>(G);
            // T_h^a[i][k] = h[k - i] (k >= i): work item = (column k, 8 of the rows)
            for (int item = ct; item < 512; item += kBwConv) {
                const int k = item & 63, r0 = (item >> 6) * 8;   // column k, rows r0 .. r0+7
                float hv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int r = r0 + q;
                    hv[q] = k >= r ? hs[k - r] : 0.f;
                }
                const uint32_t kb = (k >> 5) * (NM * 128);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float hi, lo;
                    split_tf32(hv[q], hi, lo);
                    const uint32_t o = kb + sw128_off(r0 + q, k & 31);
                    *reinterpret_cast<float *>(smem + SM::TB + d.tab * SM::BSLOT + SM::T_BHI + o) = hi;
                    *reinterpret_cast<float *>(smem + SM::TB + d.tab * SM::BSLOT + SM::T_BLO + o) = lo;
                }
            }
            const float4 *Ou = reinterpret_cast<const float4 *>(G + (Tab::B_OU - Tab::B_H));
            float4 *sOu = reinterpret_cast<float4 *>(T + SM::S_OU);
            for (int idx = ct; idx < kL * MB / 4; idx += kBwConv) sOu[idx] = Ou[idx];
            const float4 *src = reinterpret_cast<const float4 *>(G + SM::G_PART0);
            float4 *dst = reinterpret_cast<float4 *>(T + SM::S_SCAN);
            for (int idx = ct; idx < (int)(Tab::scan_bytes(F64) / 16); idx += kBwConv) dst[idx] = src[idx];
            float *coef = reinterpret_cast<float *>(T + SM::S_COEF);   // a[0..MB) | b[0..MB]
            const float *gc = reinterpret_cast<const float *>(G + SM::G_COEF);
            if (ct < 2 * MB + 1) coef[ct] = gc[ct];
            fence_proxy_async_smem();   // B is read by the tensor cores
        };
        // gy tile of `d` -> stage s
        auto issue_gy = [&](const TileDesc &d, int s) {
            if (tma_gy) {
                if (ct == 0) {
                    mbar_arrive_expect_tx(&load_bar[s], kTileBytes);
                    const int row = (int)(d.tstart / kL);
                    tma_load_3d(sbase + stage_hi(s), &tmg, 0, 0, row, &load_bar[s]);
                    tma_load_3d(sbase + stage_hi(s) + kKBlock, &tmg, 0, 1, row, &load_bar[s]);
                }
            } else {
                load_tile_async<kBwConv>(sbase + stage_hi(s), gy, d.tstart, d.tlen,
                                              gy_al && ((d.tstart & 3) == 0), ct);
            }
        };

        if (ct == 0) {
            // every slot starts as an end marker: the MMA warp ends both epilogue
            // groups (indices E and E+1) when the work runs out at index E
            for (int j = 0; j < 8; ++j) ring[j].ch = -1;
            TileDesc d0, d1;
            next_desc(d0);
            next_desc(d1);
            ring[0] = d0;
            ring[1] = d1;
            if (d0.ch >= 0) prefetch_record(d0);
        }
        named_sync(kNamedConv, kBwConv);
        int64_t issued_upto = -1;   // last tile whose gy load this thread has issued
        int64_t waited_upto = -1;   // thread 0: last tile whose gy load it saw land
        uint32_t stg_par = 0;       // parity of the next staging completion
        bool conv_alive = true;
        {
            const TileDesc d0 = ring[0], d1 = ring[1];
            if (d0.ch >= 0) {
                if (ct == 0) {
                    conv_ok[3] = wait1(stg_bar, stg_par) ? 1 : 0;
                    stg_pending = conv_ok[3] == 0;
                }
                stg_par ^= 1u;
                named_sync(kNamedConv, kBwConv);
                conv_alive = conv_ok[3] != 0;
                if (conv_alive) {
                    build_tables(d0);
                    issue_gy(d0, 0);
                    issued_upto = 0;
                    if (d1.ch >= 0) {   // its tables (if it starts a channel) wait for MMA(0)
                        issue_gy(d1, 1);
                        issued_upto = 1;
                    }
                }
            }
        }
        for (int64_t i = 0; conv_alive; ++i) {
            const int s = (int)(i % kBwNS);
            const uint32_t ph = (uint32_t)((i / kBwNS) & 1);
            const TileDesc d = ring[i & 7];
            if (d.ch < 0) {
                if (ct == 0) mbar_arrive(&full[s]);   // end marker for the MMA warp
                break;
            }
            // tile i+1 starts a channel (its descriptor is re-read where needed: the ring
            // slot is not rewritten before iteration i+7)
            const bool new1 = ring[(i + 1) & 7].ch >= 0 && ring[(i + 1) & 7].first;
            // (1) tile i+2's descriptor and (for a new channel at i+1) the record prefetch,
            //     while gy tile i lands; operand slot i&1 free once MMA(i-2), its previous
            //     reader, is done.  The descriptor's ring slot held tile i-6, read by every
            //     role once MMA(i-2) is done.  (An end marker at index E is followed by one
            //     at E+1, the other group's end, written in the same way one tile later.)
            if (ct == 0) {
                if (new1) prefetch_record(ring[(i + 1) & 7]);
                TileDesc nd;
                next_desc(nd);
                bool ok = true;
                if (tma_gy) ok = wait1(&load_bar[s], ph);
                if (ok) waited_upto = i;
                if (ok && i >= 2) ok = wait1(&mma_done[(i - 2) & 3], (uint32_t)(((i - 2) >> 2) & 1));
                ring[(i + 2) & 7] = nd;
                conv_ok[1] = ok ? 1 : 0;
            }
            if (!tma_gy) {
                if (issued_upto > i) cp_async_wait_1();
                else cp_async_wait_all();
            }
            named_sync(kNamedConv, kBwConv);
            if (!conv_ok[1]) break;
            // (2) the operand into TMEM slot i&1 (warp w: rows 32w .. 32w+31)
            tc_fence_after();
            a_to_tmem(warp, d.tlen, s, (int)(i & 1));
            named_sync(kNamedConv, kBwConv);
            if (ct == 0) mbar_arrive(&full[s]);
            // (3) gy tile i+2 into the stage just converted; then, if tile i+1 starts a
            //     channel, its tables, once the channel two back (same slot) is finished
            const TileDesc dn2 = ring[(i + 2) & 7];
            if (dn2.ch >= 0) {
                issue_gy(dn2, (int)((i + 2) % kBwNS));
                issued_upto = i + 2;
            }
            if (new1) {
                const TileDesc dn1 = ring[(i + 1) & 7];
                if (ct == 0) {
                    bool ok = true;
                    if (dn1.seq >= 2) ok = wait1(&tab_free[dn1.tab], (uint32_t)(((dn1.seq >> 1) - 1) & 1));
                    if (ok) {
                        ok = wait1(stg_bar, stg_par);
                        stg_pending = !ok;
                    }
                    conv_ok[2] = ok ? 1 : 0;
                }
                stg_par ^= 1u;
                named_sync(kNamedConv, kBwConv);
                if (!conv_ok[2]) break;
                build_tables(dn1);
            }
        }
        // a failed wait can leave copies in flight: let them land before the CTA exits
        if (ct == 0) {
            if (tma_gy)
                for (int64_t j = waited_upto + 1; j <= issued_upto; ++j)
                    mbar_wait_bounded(&load_bar[j % kBwNS], (uint32_t)((j / kBwNS) & 1), kDefaultWaitLimit);
            if (stg_pending) mbar_wait_bounded(stg_bar, stg_par, kDefaultWaitLimit);
        }
    } else if (warp == kBwMmaWarp) {
        // ============================ MMA issuer ============================
        bool issued = false;
        for (int64_t i = 0;; ++i) {
            const int s = (int)(i % kBwNS);                  // gy stage
            const uint32_t ph = (uint32_t)((i / kBwNS) & 1);
            const int pl = (int)(i & 1);                      // A_lo slot
            int ok = 1;
            if (lane == 0) ok = wait1(&full[s], ph) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            const TileDesc d = ring[i & 7];
            const int tb = (int)(i & 3);   // TMEM accumulator buffer
            const uint32_t tpar = (uint32_t)((i >> 2) & 1);
            // accumulator buffer free (its group done with tile i-4); end markers wait
            // too, or their arrivals could complete a second phase of mma_done before the
            // group has observed the previous one (a parity wait cannot tell them apart)
            if (lane == 0 && i >= 4) ok = wait1(&tmem_free[tb], tpar ^ 1u) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            if (d.ch < 0) {
                // end markers for both groups: index i for group i & 1, i+1 for the other
                if (lane == 0) {
                    mbar_arrive(&mma_done[tb]);
                    mbar_arrive(&mma_done[tb]);
                    const int tb1 = (int)((i + 1) & 3);
                    bool ok2 = true;
                    if (i + 1 >= 4) ok2 = wait1(&tmem_free[tb1], (uint32_t)((((i + 1) >> 2) & 1) ^ 1u));
                    if (ok2) {
                        mbar_arrive(&mma_done[tb1]);
                        mbar_arrive(&mma_done[tb1]);
                    }
                }
                break;
            }
            if (lane == 0) {
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(tb * 64);
#pragma unroll
                for (int kr = 0; kr < kL / 8; ++kr) {
                    // T_h^a is upper triangular: samples 8kk .. 8kk+7 reach outputs
                    // n < 8kk+8 only, so this K step covers B rows (and D columns) below
                    // 16 ceil((kk+1)/2); K runs downwards so that the widest step (all
                    // 64 columns) is the first, the one that overwrites the accumulator
                    const int kk = kL / 8 - 1 - kr;
                    const int nn = 16 * ((kk + 2) / 2);
                    const uint32_t idn = idesc_tf32_m128(nn);
                    const uint32_t kb = (kk >> 2) * (NM * 128) + (kk & 3) * 32;
                    const uint32_t ahi = tmem + ahi_col(pl) + 8 * kk;
                    const uint64_t bhi = sdesc_sw128(sbase + SM::TB + d.tab * SM::BSLOT + SM::T_BHI + kb);
                    mma_tf32_tmem_a(d_tmem, ahi, bhi, idn, kr > 0 ? 1u : 0u);
                    if (three) {
                        const uint64_t blo = sdesc_sw128(sbase + SM::TB + d.tab * SM::BSLOT + SM::T_BLO + kb);
                        mma_tf32_tmem_a(d_tmem, ahi, blo, idn, 1u);
                        mma_tf32_tmem_a(d_tmem, tmem + alo_col(pl) + 8 * kk, bhi, idn, 1u);
                    }
                }
                mma_commit(&mma_done[tb]);
                mbar_arrive(&mma_done[tb]);
            }
            issued = true;
            if (bt.stall_drill) {
                if (lane == 0) wait1(dead, 0);
                __syncwarp();
                break;
            }
        }
        if (lane == 0 && issued) {
            mma_commit(drain);
            mbar_wait_bounded(drain, 0, kDefaultWaitLimit);
        }
        __syncwarp();
    } else {
        // ====================== epilogue (two groups) =======================
        const int eg = (warp - kEpiWarp0) >> 2;            // group: tiles i with i & 1 == eg
        const int ew = (warp - kEpiWarp0) & 3;             // TMEM lane quarter (warp % 4)
        const int et = tid - (kEpiWarp0 + 4 * eg) * 32;    // chunk = TMEM lane
        const int bar_id = kNamedEpi + eg;
        volatile int *epi_ok = reinterpret_cast<volatile int *>(smem + SM::M_OK + 16 + 16 * eg);
        float *wt = reinterpret_cast<float *>(smem + SM::M_WT) + eg * 4 * MB;
        const uint32_t lane_off = (uint32_t)(ew * 32) << 16;
        const int xj = eg;   // this group's x buffer
        // a tile's x into the group's buffer (TMA by one thread, or cp.async by all)
        auto issue_x = [&](const TileDesc &d) {
            if (tma_x) {
                if (et == 0) {
                    mbar_arrive_expect_tx(&x_bar[xj], kTileBytes);
                    const int row = (int)(d.tstart / kL);
                    tma_load_3d(sbase + xbuf(xj), &tmx, 0, 0, row, &x_bar[xj]);
                    tma_load_3d(sbase + xbuf(xj) + kKBlock, &tmx, 0, 1, row, &x_bar[xj]);
                }
            } else {
                load_tile_async<128>(sbase + xbuf(xj), x, d.tstart, d.tlen,
                                     x_al && ((d.tstart & 3) == 0), et);
                cp_async_mbar_arrive_noinc(&x_bar[xj]);
            }
        };
        int64_t x_pending = -1;   // tile whose x load is issued but not yet waited for
        for (int64_t i = eg;; i += 2) {
            const int s = (int)(i & 1);   // == eg
            const int tb = (int)(i & 3);  // TMEM accumulator buffer
            // TMA x of a later tile: issued before the accumulator wait (the descriptor is
            // in the ring since the group saw MMA(i-2) done), once the previous tile's
            // grad_x store has read the buffer; the first tile and cp.async x: below
            if (et == 0) {
                if (tma_x && i > eg) {
                    const TileDesc nx = ring[i & 7];
                    bulk_wait_read0();
                    if (nx.ch >= 0) {
                        issue_x(nx);
                        x_pending = i;
                    }
                }
                epi_ok[0] = wait1(&mma_done[tb], (uint32_t)((i >> 2) & 1)) ? 1 : 0;
            }
            named_sync(bar_id, 128);
            if (!epi_ok[0]) break;
            tc_fence_after();
            const TileDesc pv = ring[i & 7];
            if (pv.ch < 0) break;
            const char *T = smem + sslot(pv.tab);
            const float *sOu = reinterpret_cast<const float *>(T + SM::S_OU);
            const float *sP = reinterpret_cast<const float *>(T + SM::S_SCAN);
            const float2 *sAt = reinterpret_cast<const float2 *>(T + SM::S_SCAN);
            const float *coef = reinterpret_cast<const float *>(T + SM::S_COEF);
            char *xs = smem + xbuf(xj);   // x tile, then grad_x (operand layout)
            if (!tma_x || i == eg) {   // (cp.async: the previous tile's plain stores have read the buffer)
                issue_x(pv);
                x_pending = i;
            }
            const int nch = (pv.tlen + kL - 1) / kL;
            const uint32_t taddr = tmem + lane_off + (uint32_t)(tb * 64);
            // the forward's state entering this chunk (read early: global latency)
            float st[MB];
            {
                const bool vch = et < nch;
                const float *src = saved + (size_t)(pv.chunk0 + et) * bt.Mstride;
#pragma unroll
                for (int m = 0; m < MB; ++m) st[m] = (vch && m < pv.M) ? src[m] : 0.f;
            }
            float E[MB];
            {
                float v[16];
                tmem_ld16(taddr, v);
                tmem_wait_ld();
#pragma unroll
                for (int m = 0; m < MB; ++m) E[m] = v[m];
            }
            // The state entering the tile from the right is the previous tile's carry
            // (always waited for, which keeps the carry barriers' phases in step).  The
            // carry chain runs through both groups tile by tile, so each group does all
            // the work that does not need it before it waits.
            float S[MB];   // S'_c = u[(c+1)L + m]
            if constexpr (!F64) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int dd = 1 << k;
                    float nx[MB];
#pragma unroll
                    for (int m = 0; m < MB; ++m) nx[m] = __shfl_down_sync(0xffffffffu, E[m], dd);
                    if (lane + dd < 32) {
                        float add[MB];
                        matvec<MB>(sP + k * MB * MB, nx, add);
#pragma unroll
                        for (int m = 0; m < MB; ++m) E[m] += add[m];
                    }
                }
                if (lane == 0) {
#pragma unroll
                    for (int m = 0; m < MB; ++m) wt[ew * MB + m] = E[m];
                }
                if (i >= 1 && et == 0)
                    epi_ok[2] = wait1(&carry_bar[s ^ 1], (uint32_t)(((i - 1) >> 1) & 1)) ? 1 : 0;
                named_sync(bar_id, 128);   // warp totals written, carry landed
                if (i >= 1 && !epi_ok[2]) break;
                float C[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) C[m] = (pv.first || i == 0) ? 0.f : carry[(s ^ 1) * MB + m];
#pragma unroll
                for (int ww = 3; ww >= 0; --ww) {
                    if (ww == ew) {
#pragma unroll
                        for (int m = 0; m < MB; ++m) S[m] = C[m];
                    }
                    float w2[MB];
                    matvec<MB>(sP + 5 * MB * MB, C, w2);
#pragma unroll
                    for (int m = 0; m < MB; ++m) C[m] = w2[m] + wt[ww * MB + m];
                }
                if (et == 0) {   // carry for the next tile (the other group)
#pragma unroll
                    for (int m = 0; m < MB; ++m) carry[s * MB + m] = C[m];
                    mbar_arrive(&carry_bar[s]);
                }
                float v[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) v[m] = S[m];
                const int e = 31 - lane;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if ((e >> k) & 1) {
                        float w2[MB];
                        matvec<MB>(sP + k * MB * MB, v, w2);
#pragma unroll
                        for (int m = 0; m < MB; ++m) v[m] = w2[m];
                    }
                }
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    const float wn = __shfl_down_sync(0xffffffffu, E[m], 1);
                    S[m] = v[m] + (lane < 31 ? wn : 0.f);
                }
                // (wt is next written in the group's next tile, several group barriers on)
            } else {
                if (i >= 1) {
                    if (et == 0) epi_ok[2] = wait1(&carry_bar[s ^ 1], (uint32_t)(((i - 1) >> 1) & 1)) ? 1 : 0;
                    named_sync(bar_id, 128);
                    if (!epi_ok[2]) break;
                }
                // serial reverse scan in double words by the whole group, from the other
                // group's carry (zero at a channel's last tile, processed first)
                float *xbuf_s = reinterpret_cast<float *>(smem + SM::SCR + eg * SM::SCR_G);
                float *sbuf = xbuf_s + kChunks * MB;
                float2 *st = reinterpret_cast<float2 *>(sbuf + kChunks * MB);   // [2][MB]
#pragma unroll
                for (int m = 0; m < MB; ++m) xbuf_s[et * MB + m] = E[m];
                if (et < MB) {
                    const bool z = pv.first || i == 0;
                    st[et] = z ? make_float2(0.f, 0.f) : carry64[(s ^ 1) * MB + et];
                }
                named_sync(bar_id, 128);
                pipe::dw_scan_group<MB>(sAt, st, xbuf_s, sbuf, nch, true, et,
                                        [&] { named_sync(bar_id, 128); });
                if (et < MB) carry64[s * MB + et] = st[(nch & 1) * MB + et];
                named_sync(bar_id, 128);
                if (et == 0) mbar_arrive(&carry_bar[s]);   // carry for the next tile
#pragma unroll
                for (int m = 0; m < MB; ++m) S[m] = et < nch ? sbuf[et * MB + m] : 0.f;
                named_sync(bar_id, 128);
            }
            // x tile landed in the group's buffer
            if (et == 0) epi_ok[1] = wait1(&x_bar[xj], (uint32_t)((i >> 1) & 1)) ? 1 : 0;
            named_sync(bar_id, 128);
            if (!epi_ok[1]) break;
            x_pending = -1;
            // samples past the channel's end read as zero: this row's tail zeroed in place
            // (only a channel's last tile has one; the row is this thread's alone)
            const int nvalid = pv.tlen - et * kL;
            if (nvalid < kL) {
#pragma unroll 1
                for (int j16 = max(nvalid, 0) >> 2; j16 < 16; ++j16) {
                    float4 *pp = reinterpret_cast<float4 *>(xs + op_piece(et, j16));
                    float4 v = *pp;
                    const int s0 = 4 * j16;
                    if (s0 + 0 >= nvalid) v.x = 0.f;
                    if (s0 + 1 >= nvalid) v.y = 0.f;
                    if (s0 + 2 >= nvalid) v.z = 0.f;
                    if (s0 + 3 >= nvalid) v.w = 0.f;
                    *pp = v;
                }
            }
            // Streamed over the chunk row, 16 columns of the adjoint at a time (u = TMEM
            // zero-state part + free response O^u S'), 4 samples per x piece: y
            // recomputed from the forward's chunk state, the lag correlations
            // grad_b[k] += u[n+k] x[n] and grad_a[k] -= u[n+1+k] y[n], and
            // grad_x = sum_k b_k u[n+k] written over x
            auto u_block = [&](int bb, float (&ub)[16]) {
                float v[16];
                tmem_ld16(taddr + bb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = bb * 16 + q;
                    float a = v[q];
#pragma unroll
                    for (int m = 0; m < MB; ++m) a = fmaf(sOu[n * MB + m], S[m], a);
                    ub[q] = a;
                }
            };
            float ucur[16], unext[16];
            u_block(0, ucur);
            if (gzi && pv.last && et == 0) {
#pragma unroll
                for (int m = 0; m < MB; ++m)
                    if (m < pv.M) gzi[pv.ch * bt.Mstride + m] = ucur[m];
            }
            float pb[MB + 1], pa[MB];
#pragma unroll
            for (int k = 0; k <= MB; ++k) pb[k] = 0.f;
#pragma unroll
            for (int k = 0; k < MB; ++k) pa[k] = 0.f;
            // low orders: the coefficients in registers (-a_1..-a_MB, b_0..b_MB), off the
            // y recursion's dependency chain; higher orders read them from shared memory
            constexpr bool kRegCoef = MB <= 8;
            float cR[kRegCoef ? 2 * MB + 1 : 1];
            if constexpr (kRegCoef) {
#pragma unroll
                for (int k = 0; k < MB; ++k) cR[k] = -coef[k];
#pragma unroll
                for (int k = 0; k <= MB; ++k) cR[MB + k] = coef[MB + k];
            }
            auto na = [&](int k) -> float {   // -a_{k+1}
                if constexpr (kRegCoef) return cR[k];
                else return -coef[k];
            };
            auto cb_ = [&](int k) -> float {   // b_k
                if constexpr (kRegCoef) return cR[MB + k];
                else return coef[MB + k];
            };
#pragma unroll 1
            for (int bb = 0; bb < kL / 16; ++bb) {
                if (bb + 1 < kL / 16) {
                    u_block(bb + 1, unext);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) unext[q] = q < MB ? S[q] : 0.f;   // u[L + m] = S'_m
                }
#define DFILT_EXT(nn) ((nn) < 16 ? ucur[(nn)] : unext[(nn) - 16])
#pragma unroll
                for (int p4 = 0; p4 < 4; ++p4) {
                    const int j16 = bb * 4 + p4;
                    const float4 xv = *reinterpret_cast<const float4 *>(xs + op_piece(et, j16));
                    const float xq[4] = {xv.x, xv.y, xv.z, xv.w};
                    float gq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int nn = 4 * p4 + q;        // within the block
                        const float xn = xq[q];
                        const float yn = fmaf(cb_(0), xn, st[0]);
#pragma unroll
                        for (int k = 0; k < MB; ++k)
                            st[k] = fmaf(na(k), yn, fmaf(cb_(1 + k), xn, k + 1 < MB ? st[k + 1] : 0.f));
#pragma unroll
                        for (int k = 0; k <= MB; ++k) pb[k] = fmaf(DFILT_EXT(nn + k), xn, pb[k]);
#pragma unroll
                        for (int k = 0; k < MB; ++k) pa[k] = fmaf(DFILT_EXT(nn + 1 + k), yn, pa[k]);
                        float g = 0.f;
#pragma unroll
                        for (int k = 0; k <= MB; ++k) g = fmaf(cb_(k), DFILT_EXT(nn + k), g);
                        gq[q] = g;
                    }
                    *reinterpret_cast<float4 *>(xs + op_piece(et, j16)) = make_float4(gq[0], gq[1], gq[2], gq[3]);
                }
#undef DFILT_EXT
#pragma unroll
                for (int q = 0; q < 16; ++q) ucur[q] = unext[q];
            }
            tc_fence_before();
            fence_proxy_async_smem();
            {
                float mine = 0.f;
#pragma unroll
                for (int k = 0; k < NACC; ++k) {
                    float v = k <= MB ? pb[k] : pa[k - MB - 1];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == k) mine = v;
                }
                // this warp's own slot (no other thread adds to it): the channel's tiles of
                // this group are summed in processing order
                if (lane < NACC) acc_ch[((pv.tab * 2 + eg) * 4 + (et >> 5)) * NACC + lane] += (double)mine;
            }
            named_sync(bar_id, 128);
            if (et == 0) mbar_arrive(&tmem_free[tb]);
            const bool tma_store = tma_gx && gx && pv.tlen == kTileSamples;
            if (tma_store) {
                if (et == 0) {
                    // asynchronous: the group's next tile waits for the read of its buffer
                    const int row = (int)(pv.tstart / kL);
                    tma_store_3d(&tmgx, 0, 0, row, sbase + xbuf(xj));
                    tma_store_3d(&tmgx, 0, 1, row, sbase + xbuf(xj) + kKBlock);
                    bulk_commit();
                }
            } else {
                if (gx) {
                    const bool al = gx_al && ((pv.tstart & 3) == 0);
#pragma unroll 4
                    for (int q = 0; q < 16; ++q) {
                        const int id = et + 128 * q;
                        const int r = id >> 4, j16 = id & 15;
                        const float4 v = *reinterpret_cast<const float4 *>(xs + op_piece(r, j16));
                        const int sidx = r * kL + j16 * 4;
                        const int nv = min(max(pv.tlen - sidx, 0), 4);
                        float *gp = gx + pv.tstart + sidx;
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
                named_sync(bar_id, 128);
            }
            // this tile's lag sums are in: count it for its channel
            if (et == 0) {
                __threadfence_block();
                atomicAdd(&tiles_done[pv.tab], 1u);
            }
            if (pv.last) {
                // the channel's other tiles (the other group's included) have added theirs
                if (et == 0) {
                    const Channel c = channel_of(bt, pv.ch);
                    const unsigned nt = (unsigned)((c.len + kTileSamples - 1) / kTileSamples);
                    volatile unsigned *cnt = tiles_done + pv.tab;
                    bool ok = false;
                    for (long long it = 0; it < bt.wait_limit; ++it) {
                        if (*cnt >= nt) {
                            ok = true;
                            break;
                        }
                        if ((it & 63) == 63) {
                            if (*abort_flag) break;
                            __nanosleep(32);
                        }
                    }
                    if (!ok && !*abort_flag) {
                        set_status(bt.status, DFILT_ERR_TIMEOUT);
                        *abort_flag = 1;
                    }
                    __threadfence_block();
                    epi_ok[3] = ok ? 1 : 0;
                }
                named_sync(bar_id, 128);
                if (!epi_ok[3]) break;
                const Channel c = channel_of(bt, pv.ch);
                for (int k = et; k < NACC; k += 128) {
                    // fixed order: warp by warp, the two groups' sums (a commutative pair: the
                    // group a tile lands on depends on the CTA's earlier channels)
                    double v = 0.0;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        double *s0 = acc_ch + ((pv.tab * 2 + 0) * 4 + w) * NACC + k;
                        double *s1 = acc_ch + ((pv.tab * 2 + 1) * 4 + w) * NACC + k;
                        v += *s0 + *s1;
                        *s0 = 0.0;
                        *s1 = 0.0;
                    }
                    if (k <= MB) {
                        if (gb && k <= c.N) gb[pv.ch * bt.Nstride + k] = (float)v;
                    } else {
                        const int m = k - MB - 1;
                        if (ga && m < c.M) ga[pv.ch * bt.Mstride + m] = (float)(-v);
                    }
                }
                if (et == 0) tiles_done[pv.tab] = 0u;
                named_sync(bar_id, 128);
                if (et == 0) mbar_arrive(&tab_free[pv.tab]);
            }
        }
        if (et == 0) {
            bulk_wait0();   // every TMA store complete before the CTA exits
            // an x load issued for a tile the group did not reach lands first
            if (tma_x && x_pending >= 0)
                mbar_wait_bounded(&x_bar[xj], (uint32_t)((x_pending >> 1) & 1), kDefaultWaitLimit);
        }
    }
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int MB, bool F64>
cudaError_t launch_bwd_ws(const float *gy, const float *x, const float *b,
                          const float *a, const float *saved, float *gx, float *gb, float *ga,
                          float *gzi, const char *tabs, unsigned long long *counter, const Batch &bt, int three, int num_sms,
                          cudaStream_t st) {
    using SM = BwSmem<MB, F64>;
    static_assert(SM::ALLOC <= pipe::kSmemMax, "shared memory budget");
    auto kern = chunk_bwd_ws_kernel<MB, F64>;
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
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const int mask = (al(gy) ? 1 : 0) | (al(x) ? 2 : 0) | ((gx && al(gx)) ? 8 : 0);
    CUtensorMap tmg, tmx, tmgx;
    std::memset(&tmg, 0, sizeof(tmg));
    std::memset(&tmx, 0, sizeof(tmx));
    std::memset(&tmgx, 0, sizeof(tmgx));
    int tma = 0;
    // tensor maps view a fixed-shape batch as rows of one chunk; a ragged batch, a
    // length that is not a whole number of chunks or a misaligned base takes cp.async
    if (!bt.offsets && bt.T % kL == 0) {
        if (make_chunk_tmap(&tmg, gy, bt.total)) tma |= 1;
        if (make_chunk_tmap(&tmx, x, bt.total)) tma |= 2;
        if (gx && make_chunk_tmap(&tmgx, gx, bt.total)) tma |= 4;
    }
    kern<<<(unsigned)grid, kBwThreads, SM::ALLOC, st>>>(gy, x, b, a, saved, gx, gb, ga, gzi, tabs, counter,
                                                       bt, three, mask, tma, tmg, tmx, tmgx); note_launch();
    return cudaGetLastError();
}

}  // namespace

template <int MB>
cudaError_t chunk_bwd_mb(const float *gy, const float *x, const float *y, const float *b,
                         const float *a, const float *saved, float *gx, float *gb, float *ga,
                         float *gzi, const char *tabs, unsigned long long *counter, const Batch &bt, bool fp64_scan, bool read_y,
                         int three, int num_sms, cudaStream_t st) {
#define ARGS gy, x, y, b, a, saved, gx, gb, ga, gzi, tabs, counter, bt, three, num_sms, st
    if constexpr (MB <= 8) {
        // warp-specialised kernel (recomputes y from the saved chunk states)
        if (!read_y) {
            if (fp64_scan) return launch_bwd_ws<MB, true>(gy, x, b, a, saved, gx, gb, ga, gzi, tabs, counter, bt, three, num_sms, st);
            return launch_bwd_ws<MB, false>(gy, x, b, a, saved, gx, gb, ga, gzi, tabs, counter, bt, three, num_sms, st);
        }
    }
    if (read_y) {
        if constexpr (MB <= 32) {
            if (fp64_scan) return launch_bwd_t<MB, true, true>(ARGS);
            if constexpr (MB <= kMaxF32ScanBucket) return launch_bwd_t<MB, false, true>(ARGS);
        }
        return cudaErrorNotSupported;
    }
    if (fp64_scan) return launch_bwd_t<MB, true, false>(ARGS);
    if constexpr (MB <= kMaxF32ScanBucket) return launch_bwd_t<MB, false, false>(ARGS);
    return cudaErrorNotSupported;
#undef ARGS
}

template cudaError_t chunk_bwd_mb<DFILT_MB>(const float *, const float *, const float *,
                                            const float *, const float *, const float *, float *,
                                            float *, float *, float *, const char *,
                                            unsigned long long *, const Batch &, bool, bool, int,
                                            int, cudaStream_t);

}  // namespace dfilt
