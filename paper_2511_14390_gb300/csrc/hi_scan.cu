// Decoupled high-order path, CUDA-core kernels: launch plan, span transitions, the
// chunk-state scan with its look-back, and the fixed-order reduction of the backward's
// per-tile lag sums.  See hi.cuh for the scheme.
#include "hi.cuh"

#ifndef DFILT_MB
#error "compile once per state bucket with -DDFILT_MB=<8|16|32|64>"
#endif

namespace dfilt {

namespace {

using hi::Plan;

// threads per state row of the scan (the CTA holds MB * TPR threads)
// (one thread per row at order 32: no shuffles, and the columns past the channel's own
// order are skipped warp-uniformly)
constexpr int scan_tpr(int mb) { return mb <= 8 ? 4 : (mb == 32 ? 1 : 2); }
// Chains (CTAs) per SM: enough warps to keep the FP32 pipes issuing, few enough that a
// long channel's chain is not slowed by many others sharing its SM (the tuning table's
// value where one is set, hi_scan_chains_default otherwise)

// ---------------------------------------------------------------------------
// Plan: per position of the launch's channel list, the tiles and scan spans before it
// (exclusive prefix sums; one block).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) hi_plan_kernel(Plan p, Batch bt) {
    __shared__ long long wt[32], ws[32];
    __shared__ long long carry_t, carry_s;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t n = hi::plan_count(p, bt);
    if (t == 0) {
        carry_t = 0;
        carry_s = 0;
    }
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + t;
        long long nt = 0, ns = 0;
        if (i < n) {
            const Channel c = channel_of(bt, hi::plan_channel(p, i, bt));
            nt = hi::tiles_of(c.len);
            ns = (nt + p.span_tiles - 1) >> p.log2_span;
        }
        // inclusive warp scans, then across warps
        long long it = nt, is = ns;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long a = __shfl_up_sync(0xffffffffu, it, o);
            const long long b = __shfl_up_sync(0xffffffffu, is, o);
            if (lane >= o) {
                it += a;
                is += b;
            }
        }
        if (lane == 31) {
            wt[warp] = it;
            ws[warp] = is;
        }
        __syncthreads();
        if (warp == 0) {
            long long a = wt[lane], b = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long a2 = __shfl_up_sync(0xffffffffu, a, o);
                const long long b2 = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) {
                    a += a2;
                    b += b2;
                }
            }
            wt[lane] = a;   // inclusive over warps
            ws[lane] = b;
        }
        __syncthreads();
        const long long offt = carry_t + (warp > 0 ? wt[warp - 1] : 0);
        const long long offs = carry_s + (warp > 0 ? ws[warp - 1] : 0);
        if (i < n) {
            p.tile_pref[i] = offt + it - nt;
            p.span_pref[i] = offs + is - ns;
        }
        __syncthreads();
        if (t == 0) {
            carry_t += wt[31];
            carry_s += ws[31];
        }
        __syncthreads();
    }
    if (t == 0) {
        p.tile_pref[n] = carry_t;
        p.span_pref[n] = carry_s;
    }
}

// Per tile and per scan span of the launch, its channel position (one warp per
// position), so that work items find their channel with one load.
__global__ void __launch_bounds__(256) hi_pos_kernel(Plan p, Batch bt) {
    const int lane = threadIdx.x & 31;
    const int64_t n = hi::plan_count(p, bt);
    for (int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * 8) {
        const int64_t t0 = p.tile_pref[i], t1 = p.tile_pref[i + 1];
        for (int64_t t = t0 + lane; t < t1; t += 32) p.tile_pos[t] = (int)i;
        const int64_t s0 = p.span_pref[i], s1 = p.span_pref[i + 1];
        for (int64_t q = s0 + lane; q < s1; q += 32) p.span_pos[q] = (int)i;
    }
}

// ---------------------------------------------------------------------------
// Span transition J = Abar^K (K = 128 * span_tiles chunks) of every channel with more
// than one span, forward (J) or adjoint (J'), from the impulse response of 1/A near
// n = 64K (hi.cuh).  One CTA per channel, the scan's thread layout; double words:
//   1. h[0 .. 64 + MB) by the all-pole difference equation (warp 0; the lanes share
//      each step's dot product)
//   2. Abar[k][m] = -sum_{l>k} a_l h[64 + k - l - m] and the impulse's state after the
//      first chunk S_1[k] = -sum_{l>k} a_l h[64 + k - l]
//   3. S_{c+1} = Abar S_c up to S_{K-1} (the one serial part: K - 2 chunk steps)
//   4. h[64(K-2) .. 64K) = the free responses of S_{K-2}, S_{K-1}:
//      h[64c + j] = sum_m h[j - m] S_c[m]
//   5. J or J' by the closed forms, column-major like the scan block
// ---------------------------------------------------------------------------
template <int MB, int TPR>
__global__ void __launch_bounds__(MB *TPR) hi_jump_kernel(HiArgs h, Batch bt, int bwd) {
    constexpr int NT = MB * TPR, JPT = MB / TPR;
    constexpr int NA = JPT >= 8 ? 4 : (JPT >= 2 ? 2 : 1);
    constexpr int H = kL + MB;   // h[0 .. H)
    extern __shared__ float4 smem4[];
    float2 *sA = reinterpret_cast<float2 *>(smem4);   // Abar, column-major [MB*MB]
    float2 *sh = sA + MB * MB;                        // h[0 .. H)
    float2 *st = sh + H;                              // [2][MB] states
    float2 *hw = st + 2 * MB;                         // h[64(K-2) .. 64K)  [128]
    float *sa = reinterpret_cast<float *>(hw + 2 * kL);   // a_1 .. a_MB
    float *red = sa + MB;                                   // [NT / 32] block sums
    const int t = threadIdx.x, r = t / TPR, p = t % TPR, lane = t & 31;
    auto sync = [] {
        if constexpr (NT == 32) __syncwarp();
        else __syncthreads();
    };
    // sum of v over the CTA, returned to every thread
    auto block_sum = [&](float v) -> float {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if constexpr (NT == 32) {
            return v;
        } else {
            if (lane == 0) red[t >> 5] = v;
            __syncthreads();
            float tot = 0.f;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) tot += red[w];
            __syncthreads();
            return tot;
        }
    };
    const int64_t pos = blockIdx.x;
    if (pos >= hi::plan_count(h.plan, bt)) return;
    const int64_t ch = hi::plan_channel(h.plan, pos, bt);
    const Channel c = channel_of(bt, ch);
    if (hi::tiles_of(c.len) <= h.plan.span_tiles) return;   // one span: no jump needed
    const int64_t K = (int64_t)kChunks << h.plan.log2_span;
    for (int k = t; k < MB; k += NT) sa[k] = k < c.M ? h.acoef[ch * bt.Mstride + k] : 0.f;
    sync();
    // 1. h by the difference equation h[n] = -sum_{j=1..MB} a_j h[n-j]
    if (t < 32) {
        if (t == 0) sh[0] = make_float2(1.f, 0.f);
        __syncwarp();
        for (int n = 1; n < H; ++n) {
            float hh = 0.f, ll = 0.f;
            for (int j = lane + 1; j <= MB; j += 32)
                if (j <= n) pipe::dw_acc(hh, ll, sh[n - j], -sa[j - 1], 0.f);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, hh, o);
                const float ol = __shfl_xor_sync(0xffffffffu, ll, o);
                const dw s2 = two_sum(hh, oh);
                hh = s2.hi;
                ll += ol + s2.lo;
            }
            if (lane == 0) {
                const dw v = fast_two_sum(hh, ll);
                sh[n] = make_float2(v.hi, v.lo);
            }
            __syncwarp();
        }
    }
    sync();
    auto H_ = [&](int n) { return n >= 0 ? sh[n] : make_float2(0.f, 0.f); };
    // 2. the chunk transition and the impulse's state after one chunk
    for (int e = t; e < MB * MB; e += NT) {
        const int k = e % MB, m = e / MB;   // element (k, m) at m*MB + k
        float hh = 0.f, ll = 0.f;
        for (int l = k + 1; l <= MB; ++l) pipe::dw_acc(hh, ll, H_(kL + k - l - m), -sa[l - 1], 0.f);
        const dw v = fast_two_sum(hh, ll);
        sA[e] = make_float2(v.hi, v.lo);
    }
    for (int k = t; k < MB; k += NT) {
        float hh = 0.f, ll = 0.f;
        for (int l = k + 1; l <= MB; ++l) pipe::dw_acc(hh, ll, H_(kL + k - l), -sa[l - 1], 0.f);
        const dw v = fast_two_sum(hh, ll);
        st[k] = make_float2(v.hi, v.lo);
    }
    sync();
    // 3. S_{c+1} = Abar S_c, c = 1 .. K-2 (S_1 in st[0]); then S_{K-2} and S_{K-1}.
    //    Forward call with a correction table: h[64c .. 64c + 64) = sum_m h[j - m] S_c[m]
    //    (the free response of the impulse's state entering chunk c, double words) goes
    //    into the table until ||S_c||_1 <= 2^-40, from where on every |h[n]| <= 2^-40
    //    max|h| (h[64c + n] = sum_m S_c[m] h[n - m]).
    // (every state bucket: the corrections' double-word sums, about 2M + N terms per
    // sample of a region, cost in proportion to the number of spans, the rescans they
    // replace in proportion to the samples; with spans long enough for the impulse
    // response to decay within half of one, they save the second pass over every span)
    const bool tab = !bwd && h.htab != nullptr && h.tcap > 0;
    const int64_t tchunks = tab ? ((int64_t)h.tcap / kL < K ? (int64_t)h.tcap / kL : K) : 0;
    float2 *ht = tab ? h.htab + (size_t)ch * h.tcap : nullptr;
    int64_t hz = -1;   // first chunk whose entering state is below the bound
    auto table_chunk = [&](int64_t cidx, const float2 *S) -> bool {   // true: bound reached
        const float nrm = block_sum(p == 0 ? fabsf(S[r].x + S[r].y) : 0.f);
        if (nrm <= 9.094947e-13f) return true;   // 2^-40
        for (int j = t; j < kL; j += NT) {
            float hh = 0.f, ll = 0.f;
            for (int m = 0; m < MB && m <= j; ++m) pipe::dw_acc(hh, ll, sh[j - m], S[m].x, S[m].y);
            const dw v = fast_two_sum(hh, ll);
            ht[cidx * kL + j] = make_float2(v.hi, v.lo);
        }
        return false;
    };
    if (tab)
        for (int j = t; j < kL; j += NT) ht[j] = sh[j];   // chunk 0: h directly
    float2 a[JPT];
#pragma unroll
    for (int q = 0; q < JPT; ++q) a[q] = sA[(p * JPT + q) * MB + r];
    int buf = 0;
    for (int64_t cc = 1; cc < K - 1; ++cc) {
        if (tab && hz < 0 && cc < tchunks && table_chunk(cc, st + buf * MB)) hz = cc;
        const float2 *cur = st + buf * MB;
        float hh[NA], ll[NA];
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            hh[i] = 0.f;
            ll[i] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < JPT; ++q) {
            const float2 sj = cur[p * JPT + q];
            pipe::dw_acc(hh[q % NA], ll[q % NA], a[q], sj.x, sj.y);
        }
        float hs = hh[0], ls = ll[0];
#pragma unroll
        for (int i = 1; i < NA; ++i) {
            const dw s2 = two_sum(hs, hh[i]);
            hs = s2.hi;
            ls += ll[i] + s2.lo;
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hs, o);
            const float ol = __shfl_xor_sync(0xffffffffu, ls, o);
            const dw s2 = two_sum(hs, oh);
            hs = s2.hi;
            ls += ol + s2.lo;
        }
        if (p == 0) {
            const dw v = fast_two_sum(hs, ls);
            st[(buf ^ 1) * MB + r] = make_float2(v.hi, v.lo);
        }
        sync();
        buf ^= 1;
    }
    // st[buf] = S_{K-1}, st[buf ^ 1] = S_{K-2}
    if (!bwd && !tab && h.hlen != nullptr && t == 0) h.hlen[ch] = 0;   // this channel rescans
    if (tab) {
        if (hz < 0 && K - 1 < tchunks && table_chunk(K - 1, st + buf * MB)) hz = K - 1;
        // samples of h kept: up to the bound when that is at most half the span; a slower
        // decay makes the corrections (double-word sums over the region, about M + N
        // multiply-adds per sample forward and backward) cost about as much as a rescan
        // (M^2 / 64 per sample), so those channels rescan (hlen 0)
        if (t == 0) h.hlen[ch] = (hz >= 0 && 2 * hz <= K) ? (int)(hz * kL) : 0;
    }
    // 4. h[64(K-2) + i], i < 128, from the free responses of the two states
    for (int i = t; i < 2 * kL; i += NT) {
        const float2 *S = st + (i < kL ? (buf ^ 1) : buf) * MB;
        const int j = i % kL;
        float hh = 0.f, ll = 0.f;
        for (int m = 0; m < MB && m <= j; ++m) pipe::dw_acc(hh, ll, sh[j - m], S[m].x, S[m].y);
        const dw v = fast_two_sum(hh, ll);
        hw[i] = make_float2(v.hi, v.lo);
    }
    sync();
    // 5. the closed forms (hw index i <-> h[64(K-2) + i], so h[64K - d] = hw[128 - d]):
    // J into h.jump, and (forward call) J' into h.jump2 for the backward
    for (int e = t; e < MB * MB; e += NT) {
        const int k = e % MB, m = e / MB;
        if (!bwd) {
            float hh = 0.f, ll = 0.f;
            for (int l = k + 1; l <= MB; ++l) pipe::dw_acc(hh, ll, hw[2 * kL + k - l - m], -sa[l - 1], 0.f);
            const dw v = fast_two_sum(hh, ll);
            h.jump[(size_t)ch * MB * MB + e] = make_float2(v.hi, v.lo);
        }
        if (bwd || h.jump2) {
            float hh = 0.f, ll = 0.f;
            for (int j = 0; j + m < MB; ++j) pipe::dw_acc(hh, ll, hw[2 * kL - 1 - k - j], -sa[j + m], 0.f);
            const dw v = fast_two_sum(hh, ll);
            (bwd ? h.jump : h.jump2)[(size_t)ch * MB * MB + e] = make_float2(v.hi, v.lo);
        }
    }
}

// ---------------------------------------------------------------------------
// Chunk-state scan.  One chain per CTA of NT = MB * TPR threads: thread (r, p) owns
// row r of the transition, columns p*JPT .. p*JPT+JPT-1 in registers (double words);
// the state vector alternates between two shared-memory buffers, one CTA barrier per
// chunk.  Part 0 of each row prefetches its entry of E kPre chunks ahead into registers
// (the chunk slots are read straight from global memory, so a CTA needs almost no
// shared memory and many chains share an SM); the output pass overwrites each slot's E
// with the chunk's state after its E was read.
// ---------------------------------------------------------------------------
template <int MB, int TPR, bool REV>
__global__ void __launch_bounds__(MB *TPR) hi_scan_kernel(HiArgs h, Batch bt) {
    using Tab = ChunkTab<MB>;
    constexpr int NT = MB * TPR, JPT = MB / TPR;
    constexpr int NA = JPT >= 8 ? 4 : (JPT >= 2 ? 2 : 1);   // independent accumulators
    constexpr int kPre = 8;                                   // E prefetch distance (chunks)
    extern __shared__ float4 smem4[];
    float2 *st = reinterpret_cast<float2 *>(smem4);                  // [2][MB]
    long long *info = reinterpret_cast<long long *>(st + 2 * MB);    // [4]
    float *ering = reinterpret_cast<float *>(info + 4);              // [kPre][MB] E prefetch
    const int t = threadIdx.x, r = t / TPR, p = t % TPR;
    auto sync = [] {
        if constexpr (NT == 32) __syncwarp();
        else __syncthreads();
    };
    const int64_t n = hi::plan_count(h.plan, bt);
    const int64_t total = h.plan.span_pref[n];
    const int ST = h.plan.span_tiles;
    const int Ms = bt.Mstride;
    float2 a[JPT];
    int64_t cur_ch = -1;
    bool first_item = true;

    for (;;) {
        if (t == 0) info[0] = (long long)atomicAdd(h.counter, 1ull);
        sync();
        const int64_t w = info[0];
        sync();   // info[] is rewritten below
        if (w >= total) break;
        const int64_t pos = h.plan.span_pos[w];
        const int64_t ch = hi::plan_channel(h.plan, pos, bt);
        const Channel c = channel_of(bt, ch);
        const int64_t s = w - h.plan.span_pref[pos];
        const int64_t nsp = h.plan.span_pref[pos + 1] - h.plan.span_pref[pos];
        const int64_t nchunks = (c.len + kL - 1) / kL;
        const int64_t sp = REV ? nsp - 1 - s : s;   // the span's index in time
        const int64_t k0 = sp * ST * kChunks;       // the span's chunks [k0, k1)
        int64_t k1 = (k0 + (int64_t)ST * kChunks < nchunks) ? k0 + (int64_t)ST * kChunks : nchunks;
        const int64_t cbase = c.off / kL + ch;       // the channel's first chunk slot
        {   // debug build: a span that fails its index checks scans no chunk
            const int64_t n0 = c.off + k0 * kL, n1 = c.off + (k1 * kL < c.len ? k1 * kL : c.len);
            if (!hi::dbg_range_ok(bt, n0, n1 - n0, cbase + k0, k1 - k0)) k1 = k0;
        }
        if (ch != cur_ch) {
            const float2 *At = reinterpret_cast<const float2 *>(h.tabs + (size_t)ch * h.tab_stride +
                                                                (REV ? Tab::B_SCAN : Tab::F_SCAN));
#pragma unroll
            for (int q = 0; q < JPT; ++q) a[q] = __ldg(At + (p * JPT + q) * MB + r);
            cur_ch = ch;
        }

        // One chunk step: the state in st[buf] enters the chunk whose input is e (this
        // row's entry, part 0 only); the next state goes to st[buf ^ 1].  With a slot, the
        // entering state is written to it.
        auto step = [&](float e, int buf, float *slot_row) {
            const float2 *cur = st + buf * MB;
            float2 *nxt = st + (buf ^ 1) * MB;
            float hh[NA], ll[NA];
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                hh[i] = 0.f;
                ll[i] = 0.f;
            }
            if (p == 0) hh[0] = e;
            if constexpr (TPR == 1) {
                // columns in blocks of 4, up to the channel's order (zero beyond)
#pragma unroll
                for (int q4 = 0; q4 < JPT; q4 += 4) {
                    if (q4 < c.M) {
#pragma unroll
                        for (int q = q4; q < q4 + 4; ++q) {
                            const float2 sj = cur[q];
                            pipe::dw_acc(hh[q % NA], ll[q % NA], a[q], sj.x, sj.y);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < JPT; ++q) {
                    const float2 sj = cur[p * JPT + q];
                    pipe::dw_acc(hh[q % NA], ll[q % NA], a[q], sj.x, sj.y);
                }
            }
            float hs = hh[0], ls = ll[0];
#pragma unroll
            for (int i = 1; i < NA; ++i) {
                const dw s2 = two_sum(hs, hh[i]);
                hs = s2.hi;
                ls += ll[i] + s2.lo;
            }
#pragma unroll
            for (int o = TPR / 2; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, hs, o);
                const float ol = __shfl_xor_sync(0xffffffffu, ls, o);
                const dw s2 = two_sum(hs, oh);
                hs = s2.hi;
                ls += ol + s2.lo;
            }
            if (p == 0) {
                if (slot_row && r < c.M) slot_row[r] = cur[r].x + cur[r].y;
                const dw v = fast_two_sum(hs, ls);
                nxt[r] = make_float2(v.hi, v.lo);
            }
            sync();
        };

        // Scan the span's chunks in processing order from the state in st[buf0]; returns
        // the buffer holding the final state.  `out` writes the states to the slots.  The
        // E entry of chunk i + kPre is copied (cp.async) into this lane's ring slot while
        // chunk i is scanned; each lane reads and refills only its own slots.
        auto run = [&](int buf0, bool out) -> int {
            int buf = buf0;
            const int64_t cnt = k1 - k0;
            const bool ld = (p == 0) && (r < c.M);
            auto slot = [&](int64_t i) {   // the i-th chunk in processing order
                return h.states + (size_t)(cbase + (REV ? k1 - 1 - i : k0 + i)) * Ms;
            };
            auto issue = [&](int64_t i) {
                if (p == 0) {
                    const bool v = ld && i < cnt;
                    cp_async4(smem_u32(ering + (i % kPre) * MB + r), v ? (const void *)(slot(i) + r)
                                                                      : (const void *)h.states,
                              v ? 4 : 0);
                }
                cp_async_commit();
            };
            for (int u = 0; u < kPre; ++u) issue(u);
#pragma unroll 1
            for (int64_t i = 0; i < cnt; ++i) {
                asm volatile("cp.async.wait_group %0;\n" ::"n"(kPre - 1) : "memory");
                const float e = p == 0 ? ering[(i % kPre) * MB + r] : 0.f;
                issue(i + kPre);
                step(e, buf, out ? slot(i) : nullptr);
                buf ^= 1;
            }
            cp_async_wait_all();
            return buf;
        };

        // timeout drill: the first item also waits on a flag nothing sets
        if (first_item && bt.stall_drill) {
            bool ok = false;
            if (t == 0) {
                volatile long long *dead = info + 3;
                *dead = 0;
                for (long long it = 0; it < bt.wait_limit; ++it) {
                    if (*dead) {
                        ok = true;
                        break;
                    }
                    if (it > 64) __nanosleep(32);
                }
                if (!ok) set_status(bt.status, DFILT_ERR_TIMEOUT);
                info[1] = ok ? 1 : 0;
            }
            sync();
            if (!info[1]) break;
        }
        first_item = false;

        int fin;
        if (s == 0) {
            // the channel's initial state: zi (forward) or zero (adjoint, App. A)
            if (t < MB) {
                const float z = (!REV && h.zi && t < c.M) ? h.zi[ch * Ms + t] : 0.f;
                st[t] = make_float2(z, 0.f);
            }
            sync();
            fin = run(0, true);
            if (nsp > 1) {
                if (t < MB) h.incl[(size_t)w * MB + t] = st[fin * MB + t];
                sync();
                if (t == 0) {
                    __threadfence();
                    hi::st_release(h.flags + w, 1u);
                }
            }
        } else {
            // aggregate: the span from a zero state.  Forward spans of channels with a
            // correction table keep these zero-start states (written to the slots) and
            // their entry state; the Y pass and hi_yfix add the entry state's free
            // response, so the span is not rescanned.
            const bool keep = h.hlen != nullptr && h.hlen[ch] > 0;
            if (t < MB) st[t] = make_float2(0.f, 0.f);
            sync();
            const int ag = run(0, keep);
            const int pb = ag ^ 1;   // the predecessor's inclusive state goes here
            if (t == 0) {
                bool ok = false;
                for (long long it = 0; it < bt.wait_limit; ++it) {
                    if (hi::ld_acquire(h.flags + (w - 1)) != 0u) {
                        ok = true;
                        break;
                    }
                    if (it > 64) __nanosleep(64);
                }
                if (!ok) set_status(bt.status, DFILT_ERR_TIMEOUT);
                __threadfence();
                info[1] = ok ? 1 : 0;
            }
            sync();
            if (!info[1]) break;
            if (t < MB) st[pb * MB + t] = hi::ld_cg2(h.incl + (size_t)(w - 1) * MB + t);
            sync();
            if (keep && t < c.M) h.entry[(size_t)w * Ms + t] = st[pb * MB + t];
            // the adjoint's time-first span without a rescan: its inclusive state is grad_zi
            const bool zi_here = REV && keep && sp == 0 && h.gzi != nullptr;
            if (s + 1 < nsp || zi_here) {
                // P_s = J P_{s-1} + A_s, published for the next span
                const float2 *J = h.jump + (size_t)ch * MB * MB;
                float hh = 0.f, ll = 0.f;
                if (p == 0) {
                    hh = st[ag * MB + r].x;
                    ll = st[ag * MB + r].y;
                }
#pragma unroll 4
                for (int q = 0; q < JPT; ++q) {
                    const float2 pj = st[pb * MB + p * JPT + q];
                    pipe::dw_acc(hh, ll, __ldg(J + (p * JPT + q) * MB + r), pj.x, pj.y);
                }
#pragma unroll
                for (int o = TPR / 2; o > 0; o >>= 1) {
                    const float oh = __shfl_xor_sync(0xffffffffu, hh, o);
                    const float ol = __shfl_xor_sync(0xffffffffu, ll, o);
                    const dw s2 = two_sum(hh, oh);
                    hh = s2.hi;
                    ll += ol + s2.lo;
                }
                if (p == 0) {
                    const dw v = fast_two_sum(hh, ll);
                    if (s + 1 < nsp) h.incl[(size_t)w * MB + r] = make_float2(v.hi, v.lo);
                    if (zi_here && r < c.M) h.gzi[ch * Ms + r] = v.hi + v.lo;
                }
                sync();
                if (t == 0 && s + 1 < nsp) {
                    __threadfence();
                    hi::st_release(h.flags + w, 1u);
                }
            }
            fin = keep ? ag : run(pb, true);
        }
        // the adjoint's last state is u[0 : MB) = grad_zi (the span holding chunk 0)
        if (REV && sp == 0 && h.gzi && t < c.M && !(s > 0 && h.hlen != nullptr && h.hlen[ch] > 0)) {
            h.gzi[ch * Ms + t] = st[fin * MB + t].x + st[fin * MB + t].y;
        }
        sync();
    }
}

// ---------------------------------------------------------------------------
// E pass on the CUDA cores: for every chunk of the launch's tiles, E_c = R_L x_c
// (forward: the zero-state end state of the chunk) or E'_c = (T_h^a G_c)[0:MB] (adjoint:
// the reversed Toeplitz product's first MB rows, h the impulse response of 1/A), into
// the chunk slots.  64 x M FMAs per chunk in FP32 (more accurate than a split-TF32
// product, and far below the FP32 rate for M <= 64): the pass streams the signal once.
// Thread = chunk row; tiles are taken from a counter in runs of eight (mostly one
// channel: the table R^T[j][m] is rebuilt in shared memory only when the channel
// changes) and staged by cp.async in two shared-memory stages, the next tile's copy in
// flight while this one is summed.  Samples past a channel's end are zero.
// ---------------------------------------------------------------------------
template <int MB>
struct ESmem {
    static constexpr uint32_t STAGE = pipe::kTileBytes;           // one 128 x 64 signal tile
    static constexpr uint32_t TAB = 2 * STAGE;                    // R^T [kL][MB] floats
    static constexpr uint32_t ITEM = TAB + (uint32_t)kL * MB * 4; // work item (8 bytes)
    static constexpr uint32_t BYTES = ITEM + 16;
};

template <int MB, bool BWD>
__global__ void __launch_bounds__(kChunks) hi_e_kernel(HiArgs h, Batch bt, int sig_al, int st_al) {
    using Tab = ChunkTab<MB>;
    using SM = ESmem<MB>;
    constexpr int kThreads = kChunks;
    extern __shared__ float4 smem4[];
    char *smem = reinterpret_cast<char *>(smem4);
    const uint32_t sbase = smem_u32(smem);
    float *tab = reinterpret_cast<float *>(smem + SM::TAB);
    long long *item = reinterpret_cast<long long *>(smem + SM::ITEM);
    const int tid = threadIdx.x;
    const int64_t n = hi::plan_count(h.plan, bt);
    const int64_t total = h.plan.tile_pref[n];
    const int Ms = bt.Mstride;
    constexpr int kRun = 8;
    int64_t w = 0, wend = 0, cur_ch = -1;
    int stage = 0;
    bool pre = false;   // this tile already in flight (copied during the previous one)
    auto tile_of = [&](int64_t wi, int64_t &ch, Channel &c, int64_t &tstart, int &tlen) {
        const int64_t pos = h.plan.tile_pos[wi];
        ch = hi::plan_channel(h.plan, pos, bt);
        c = channel_of(bt, ch);
        const int64_t tile = wi - h.plan.tile_pref[pos];
        tstart = c.off + tile * kTileSamples;
        const int64_t tl = c.len - tile * kTileSamples;
        tlen = (int)(tl < kTileSamples ? tl : kTileSamples);
        // debug build: a tile that fails its index checks is empty
        if (!hi::dbg_range_ok(bt, tstart, tlen, c.off / kL + ch + (tstart - c.off) / kL, (tlen + kL - 1) / kL))
            tlen = 0;
    };
    for (;;) {
        if (w >= wend) {
            if (tid == 0) *item = (long long)atomicAdd(h.counter, 1ull);
            __syncthreads();
            w = *item * kRun;
            __syncthreads();   // *item is rewritten at the next run
            if (w >= total) break;
            wend = w + kRun < total ? w + kRun : total;
        }
        int64_t ch, tstart;
        Channel c;
        int tlen;
        tile_of(w, ch, c, tstart, tlen);
        const int nch = (tlen + kL - 1) / kL;
        const int64_t slot0 = c.off / kL + ch + (tstart - c.off) / kL;   // the tile's first chunk slot
        if (!pre)
            pipe::load_tile_async<kThreads>(sbase + stage * SM::STAGE, h.sig, tstart, tlen,
                                            sig_al && ((tstart & 3) == 0), tid);
        const bool has_next = w + 1 < wend;
        if (has_next) {
            int64_t nch_, ntstart;
            Channel nc;
            int ntlen;
            tile_of(w + 1, nch_, nc, ntstart, ntlen);
            pipe::load_tile_async<kThreads>(sbase + (stage ^ 1) * SM::STAGE, h.sig, ntstart, ntlen,
                                            sig_al && ((ntstart & 3) == 0), tid);
        }
        if (ch != cur_ch) {
            // R^T[j][m]: forward R_L[m][j]; adjoint h[j - m] for j >= m (else 0)
            const char *R = h.tabs + (size_t)ch * h.tab_stride;
            for (int idx = tid; idx < kL * MB; idx += kThreads) {
                const int j = idx / MB, m = idx % MB;
                float v;
                if constexpr (BWD) v = j >= m ? reinterpret_cast<const float *>(R + Tab::B_H)[j - m] : 0.f;
                else v = reinterpret_cast<const float *>(R + Tab::F_RL)[m * kL + j];
                tab[idx] = v;
            }
            cur_ch = ch;
        }
        if (has_next) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        else cp_async_wait_all();
        __syncthreads();
        if (tid < nch) {
            const char *xs = smem + stage * SM::STAGE;
            float acc[MB];
#pragma unroll
            for (int m = 0; m < MB; ++m) acc[m] = 0.f;
#pragma unroll 1
            for (int j16 = 0; j16 < 16; ++j16) {
                const float4 xv = *reinterpret_cast<const float4 *>(xs + pipe::op_piece(tid, j16));
                const float xq[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float *tr = tab + (j16 * 4 + q) * MB;
#pragma unroll
                    for (int m4 = 0; m4 < MB; m4 += 4) {
                        if (m4 < c.M) {   // rows past the channel's order are not needed
                            const float4 t4 = *reinterpret_cast<const float4 *>(tr + m4);
                            acc[m4] = fmaf(t4.x, xq[q], acc[m4]);
                            acc[m4 + 1] = fmaf(t4.y, xq[q], acc[m4 + 1]);
                            acc[m4 + 2] = fmaf(t4.z, xq[q], acc[m4 + 2]);
                            acc[m4 + 3] = fmaf(t4.w, xq[q], acc[m4 + 3]);
                        }
                    }
                }
            }
            float *dst = h.states + (size_t)(slot0 + tid) * Ms;
            if (st_al) {
#pragma unroll
                for (int m4 = 0; m4 < MB; m4 += 4) {
                    if (m4 + 4 <= c.M) {
                        *reinterpret_cast<float4 *>(dst + m4) =
                            make_float4(acc[m4], acc[m4 + 1], acc[m4 + 2], acc[m4 + 3]);
                    } else if (m4 < c.M) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (m4 + i < c.M) dst[m4 + i] = acc[m4 + i];
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < MB; ++m)
                    if (m < c.M) dst[m] = acc[m];
            }
        }
        __syncthreads();   // this stage and the table are free again
        stage ^= 1;
        ++w;
        pre = has_next;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// Lag sums of the coefficient gradients per tile, from the U pass's zero-start adjoint u
// (adjoint correction: hi_ufix_kernel):  b-lag k = sum_n u_ext[n + k] x[n] (k = 0..N),
// a-lag k = sum_n u_ext[n + k] y[n] (k = 1..M), per 64-sample chunk row with the row's
// extension u_ext[64 + m] = S'_c[m] (the adjoint chunk state: the next chunk's first
// values from the same span).  A tile is taken in two halves of 64 rows staged in shared
// memory (rows padded to odd strides); thread = (row, block of 16 lags) for the blocks
// the channel's orders need, the 16 products of a sample from a sliding register window
// over u, both halves accumulated per thread; warp trees over the 32 rows of a warp and
// the two warps of a block in a fixed order give the tile's partial (the same layout as
// before: b-lags at 0..MB, a-lag k at MB + k).
// ---------------------------------------------------------------------------
template <int MB>
struct LagSmem {
    static constexpr int UROW = kL + MB + 16 + 1;   // u row + tail + window slack, odd
    static constexpr int XROW = kL + 1;
    static constexpr int NBLK = (MB + 1 + 15) / 16 + (MB + 15) / 16;   // lag blocks, at most
    float u[64 * UROW];
    float x[64 * XROW];
    float y[64 * XROW];
    float red[NBLK][2][16];
    long long item;
};

template <int MB>
__global__ void __launch_bounds__(256) hi_lag_kernel(HiArgs h, Batch bt) {
    using SM = LagSmem<MB>;
    constexpr int NT = 256, NACC = hi::nacc<MB>();
    constexpr int UPT = (64 * SM::NBLK + NT - 1) / NT;   // units per thread, at most
    extern __shared__ float4 smem4[];
    SM &sm = *reinterpret_cast<SM *>(smem4);
    const int t = threadIdx.x, lane = t & 31;
    const int64_t n = hi::plan_count(h.plan, bt);
    const int64_t total = h.plan.tile_pref[n];
    const int Ms = bt.Mstride;
    constexpr int kRun = 1;   // no per-channel tables here: tiles one at a time balance best
    int64_t w = 0, wend = 0;
    for (;;) {
        if (w >= wend) {
            if (t == 0) sm.item = (long long)atomicAdd(h.counter, 1ull);
            __syncthreads();
            w = sm.item * kRun;
            __syncthreads();
            if (w >= total) break;
            wend = w + kRun < total ? w + kRun : total;
        }
        const int64_t pos = h.plan.tile_pos[w];
        const int64_t ch = hi::plan_channel(h.plan, pos, bt);
        const Channel c = channel_of(bt, ch);
        const int64_t tile = w - h.plan.tile_pref[pos];
        const int64_t tstart = c.off + tile * kTileSamples;
        const int64_t tl = c.len - tile * kTileSamples;
        int tlen = (int)(tl < kTileSamples ? tl : kTileSamples);
        int nch = (tlen + kL - 1) / kL;
        const int64_t slot0 = c.off / kL + ch + tile * kChunks;
        // debug build: a tile that fails its index checks is empty (its partial is zero)
        if (!hi::dbg_range_ok(bt, tstart, tlen, slot0, nch)) {
            tlen = 0;
            nch = 0;
        }
        const int nbx = (c.N + 1 + 15) / 16, nby = (c.M + 15) / 16, nblk = nbx + nby;
        const int units = 64 * nblk;
        float acc[UPT][16];
#pragma unroll
        for (int q = 0; q < UPT; ++q)
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[q][j] = 0.f;
        for (int hf = 0; hf < 2 && 64 * hf < nch; ++hf) {
            __syncthreads();   // the previous half's rows are no longer read
            // stage rows 64 hf .. 64 hf + 63: u, x, y (zero past the tile's samples), the
            // tail of each u row from the adjoint chunk state, zeros beyond
            // (4-byte async copies: the rows are padded to odd strides; zero-filled)
            const uint32_t su = smem_u32(sm.u), sx = smem_u32(sm.x), sy = smem_u32(sm.y);
#pragma unroll 4
            for (int e = t; e < 64 * kL; e += NT) {
                const int r = e / kL, i = e % kL;
                const int sidx = (64 * hf + r) * kL + i;
                const int nb = sidx < tlen ? 4 : 0;
                const int64_t gi = tstart + (nb ? sidx : 0);
                cp_async4(su + 4 * (r * SM::UROW + i), h.ubuf + gi, nb);
                cp_async4(sx + 4 * (r * SM::XROW + i), h.x + gi, nb);
                cp_async4(sy + 4 * (r * SM::XROW + i), h.y + gi, nb);
            }
            for (int e = t; e < 64 * (MB + 16); e += NT) {
                const int r = e / (MB + 16), m = e % (MB + 16);
                const int row = 64 * hf + r;
                const bool v = m < c.M && row < nch;
                cp_async4(su + 4 * (r * SM::UROW + kL + m), h.states + (v ? (size_t)(slot0 + row) * Ms + m : 0),
                          v ? 4 : 0);
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
#pragma unroll
            for (int q = 0; q < UPT; ++q) {
                const int uidx = t + NT * q;
                if (uidx < units) {   // uniform over each warp (units is a multiple of 64)
                    const int blk = uidx / 64, r = uidx % 64;
                    const bool xb = blk < nbx;
                    const int lag0 = xb ? 16 * blk : 16 * (blk - nbx) + 1;
                    const float *src = (xb ? sm.x : sm.y) + r * SM::XROW;
                    const float *ur = sm.u + r * SM::UROW + lag0;
                    float win[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) win[j] = ur[j];
#pragma unroll 16
                    for (int i = 0; i < kL; ++i) {
                        const float v = src[i];
#pragma unroll
                        for (int j = 0; j < 16; ++j) acc[q][j] = fmaf(win[j], v, acc[q][j]);
#pragma unroll
                        for (int j = 0; j < 15; ++j) win[j] = win[j + 1];
                        win[15] = ur[i + 16];
                    }
                }
            }
        }
        // per block: the 32 rows of each warp in a fixed tree, then the block's two warps
#pragma unroll
        for (int q = 0; q < UPT; ++q) {
            const int uidx = t + NT * q;
            if (uidx < units) {
                const int blk = uidx / 64, wh = (uidx % 64) >> 5;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float v = acc[q][j];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) sm.red[blk][wh][j] = v;
                }
            }
        }
        __syncthreads();
        for (int k = t; k < NACC; k += NT) {
            float v = 0.f;
            if (k <= MB) {   // b-lag k
                if (k <= c.N) v = sm.red[k / 16][0][k % 16] + sm.red[k / 16][1][k % 16];
            } else {         // a-lag k - MB
                const int lg = k - MB, blk = nbx + (lg - 1) / 16, j = (lg - 1) % 16;
                if (lg <= c.M) v = sm.red[blk][0][j] + sm.red[blk][1][j];
            }
            h.partial[(size_t)w * NACC + k] = v;
        }
        ++w;
    }
}

// ---------------------------------------------------------------------------
// Entry-state correction of y (forward, and the backward's recomputed y): for every
// span s > 0 of a channel with a correction table, y[n] += sum_{m<M} P_m h[n - m] over
// the span's first hlen + M - 1 samples (n from the span start, h[j] = 0 for j < 0 and,
// below 2^-40 of its largest value, for j >= hlen), in double words (P and h are kept as
// double words; the sum cancels heavily for ill-conditioned filters).  One CTA per span
// at a time; h in shared memory 1024 samples at a time, four samples per thread, the sum
// over m in a fixed order.
// ---------------------------------------------------------------------------
template <int MB>
__global__ void __launch_bounds__(256) hi_yfix_kernel(HiArgs h, Batch bt) {
    constexpr int kBlk = 1024;
    __shared__ float2 hs[kBlk + MB];
    __shared__ float2 P[MB];
    const int t = threadIdx.x;
    const int64_t n = hi::plan_count(h.plan, bt);
    const int64_t items = h.plan.span_pref[n];
    const int64_t span_len = (int64_t)h.plan.span_tiles * kTileSamples;
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const int64_t pos = h.plan.span_pos[w];
        const int64_t sp = w - h.plan.span_pref[pos];
        if (sp == 0) continue;
        const int64_t ch = hi::plan_channel(h.plan, pos, bt);
        const int hl = h.hlen[ch];
        if (hl <= 0) continue;
        const Channel c = channel_of(bt, ch);
        const int64_t s0 = sp * span_len;
        const int64_t slen = c.len - s0 < span_len ? c.len - s0 : span_len;
        const int64_t want = (int64_t)hl + c.M - 1;
        int64_t rlen = want < slen ? want : slen;
        if (!hi::dbg_range_ok(bt, c.off + s0, rlen, 0, 0)) rlen = 0;   // debug build: skip
        __syncthreads();   // the previous span's P and h are no longer read
        if (t < MB) P[t] = t < c.M ? h.entry[(size_t)w * bt.Mstride + t] : make_float2(0.f, 0.f);
        const float2 *hc = h.htab + (size_t)ch * h.tcap;
        float *yp = h.out + c.off + s0;
        for (int64_t b0 = 0; b0 < rlen; b0 += kBlk) {
            __syncthreads();
            for (int i = t; i < kBlk + MB - 1; i += 256) {   // hs[i] = h[b0 - (MB - 1) + i]
                const int64_t j = b0 - (MB - 1) + i;
                hs[i] = (j >= 0 && j < hl) ? hc[j] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            // the thread's four samples t + 256 q as four independent chains (each
            // sample still sums its terms in the order m = 0, 1, ...)
            constexpr int Q = kBlk / 256;
            float hh[Q], ll[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                hh[q] = 0.f;
                ll[q] = 0.f;
            }
#pragma unroll 4
            for (int m = 0; m < MB; ++m) {
                if (m < c.M) {
                    const float2 pm = P[m];
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const float2 hv = hs[t + 256 * q + MB - 1 - m];
                        pipe::dw_acc(hh[q], ll[q], pm, hv.x, hv.y);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int i = t + 256 * q;
                if (b0 + i < rlen) yp[b0 + i] += hh[q] + ll[q];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Entry-state correction of the adjoint (backward, hi.cuh): for every span of a channel
// with a table except its last in time, with P' its adjoint entry state and i the
// reversed-time offset from its last sample (sample n = end - 1 - i):
//   w_j = -sum_{k=j+1..M} a_k P'_{k-j-1}                        (j < M, double words)
//   v[i] = sum_{j<M} h[i - j] w_j,  v[-1-m] = P'_m               (double words)
//   grad_x[n] += sum_{k<=N} b_k v[i - k]                          (double words)
//   lag sums: b-lag k += v[i - k] x[n],  a-lag k += v[i - k] y[n]   (FP32, per thread)
// over i < min(hlen + 3 MB, span length) (v vanishes below 2^-40 of its scale beyond
// hlen + M - 1).  One CTA per span at a time, 1024 samples per block step; the lag sums
// are reduced in a fixed order into the span's partial.
// ---------------------------------------------------------------------------
template <int MB>
__global__ void __launch_bounds__(256) hi_ufix_kernel(HiArgs h, Batch bt) {
    constexpr int kBlk = 1024, NT = 256, NACC = hi::nacc<MB>();
    __shared__ float2 hs[kBlk + MB];        // h[b0 - (MB - 1) + q]
    __shared__ float2 vs[2][kBlk + MB];     // v[b0 - MB + q], double buffered across blocks
    __shared__ float2 W[MB], P[MB];
    __shared__ float Bk[MB + 1];
    __shared__ float red[NT / 32][NACC];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t n = hi::plan_count(h.plan, bt);
    const int64_t items = h.plan.span_pref[n];
    const int64_t span_len = (int64_t)h.plan.span_tiles * kTileSamples;
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const int64_t pos = h.plan.span_pos[w];
        const int64_t s = w - h.plan.span_pref[pos];   // processing index (last in time first)
        if (s == 0) continue;
        const int64_t ch = hi::plan_channel(h.plan, pos, bt);
        const int hl = h.hlen[ch];
        if (hl <= 0) continue;
        const Channel c = channel_of(bt, ch);
        const int64_t nsp = h.plan.span_pref[pos + 1] - h.plan.span_pref[pos];
        const int64_t end = (nsp - s) * span_len;       // a full span ends here
        const int64_t want = (int64_t)hl + 3 * MB;
        int64_t R = want < span_len ? want : span_len;
        if (!hi::dbg_range_ok(bt, c.off + end - R, R, 0, 0)) R = 0;   // debug build: skip
        __syncthreads();   // the previous span's shared data is no longer read
        if (t < MB) P[t] = t < c.M ? h.entry[(size_t)w * bt.Mstride + t] : make_float2(0.f, 0.f);
        __syncthreads();
        if (t < MB) {
            float hh = 0.f, ll = 0.f;
            for (int k = t + 1; k <= c.M; ++k) pipe::dw_acc(hh, ll, P[k - t - 1], -h.acoef[ch * bt.Mstride + k - 1], 0.f);
            const dw v = fast_two_sum(hh, ll);
            W[t] = t < c.M ? make_float2(v.hi, v.lo) : make_float2(0.f, 0.f);
            // the first block's halo: v[-1 - m] = P'_m
            vs[0][MB - 1 - t] = P[t];
        }
        if (t <= MB) Bk[t] = t <= c.N ? h.bcoef[ch * bt.Nstride + t] : 0.f;
        float acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[k] = 0.f;
        const float2 *hc = h.htab + (size_t)ch * h.tcap;
        const float *xp = h.x + c.off + end - 1, *yp = h.y + c.off + end - 1;   // minus i
        float *gp = h.out ? h.out + c.off + end - 1 : nullptr;
        int cur = 0;
        for (int64_t b0 = 0; b0 < R; b0 += kBlk) {
            for (int q = t; q < kBlk + MB - 1; q += NT) {
                const int64_t j = b0 - (MB - 1) + q;
                hs[q] = (j >= 0 && j < hl) ? hc[j] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            // v over this block into vs[cur][MB + q]: the thread's four samples q = t + NT e
            // as four independent chains (each sums in the order j = 0, 1, ...)
            constexpr int Q = kBlk / NT;
            {
                float hh[Q], ll[Q];
#pragma unroll
                for (int e = 0; e < Q; ++e) {
                    hh[e] = 0.f;
                    ll[e] = 0.f;
                }
#pragma unroll 4
                for (int j = 0; j < MB; ++j) {
                    if (j < c.M) {
                        const float2 wj = W[j];
#pragma unroll
                        for (int e = 0; e < Q; ++e) {
                            const float2 hv = hs[t + NT * e + MB - 1 - j];
                            pipe::dw_acc(hh[e], ll[e], wj, hv.x, hv.y);
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < Q; ++e) {
                    const int q = t + NT * e;
                    const dw v = b0 + q < R ? fast_two_sum(hh[e], ll[e]) : dw{0.f, 0.f};
                    vs[cur][MB + q] = make_float2(v.hi, v.lo);
                }
            }
            __syncthreads();
            // grad_x of this block's samples (the thread's four as independent chains, each
            // in the order k = 0, 1, ...), then the lag sums sample by sample
            float gh[Q], gl[Q];
#pragma unroll
            for (int e = 0; e < Q; ++e) {
                gh[e] = 0.f;
                gl[e] = 0.f;
            }
#pragma unroll 4
            for (int k = 0; k <= MB; ++k) {
                if (k <= c.N) {
                    const float2 bk = make_float2(Bk[k], 0.f);
#pragma unroll
                    for (int e = 0; e < Q; ++e) {
                        const float2 vk = vs[cur][MB + t + NT * e - k];
                        pipe::dw_acc(gh[e], gl[e], bk, vk.x, vk.y);
                    }
                }
            }
#pragma unroll 1
            for (int e = 0; e < Q; ++e) {
                const int q = t + NT * e;
                const int64_t i = b0 + q;
                if (i >= R) break;
                const float2 *vq = &vs[cur][MB + q];   // vq[-k] = v[i - k]
                if (h.out) gp[-i] += gh[e] + gl[e];
                const float xv = xp[-i], yv = yp[-i];
#pragma unroll
                for (int k = 0; k <= MB; ++k) {
                    const float vf = vq[-k].x + vq[-k].y;
                    acc[k] = fmaf(vf, xv, acc[k]);
                    if (k >= 1) acc[MB + k] = fmaf(vf, yv, acc[MB + k]);
                }
            }
            __syncthreads();
            // the next block's halo: v[b0 + kBlk - MB .. b0 + kBlk)
            if (t < MB) vs[cur ^ 1][t] = vs[cur][kBlk + t];
            cur ^= 1;
        }
        // the span's lag sums, fixed order: warp trees, then warps 0..7
#pragma unroll
        for (int k = 0; k < NACC; ++k) {
            float v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        for (int k = t; k < NACC; k += NT) {
            float v = 0.f;
#pragma unroll
            for (int e = 0; e < NT / 32; ++e) v += red[e][k];
            h.span_part[(size_t)w * NACC + k] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Coefficient gradients: per channel, the tiles' lag sums in tile order (FP64).
// One warp per channel position.
// ---------------------------------------------------------------------------
template <int MB>
__global__ void __launch_bounds__(128) hi_reduce_kernel(HiArgs h, Batch bt) {
    constexpr int NACC = hi::nacc<MB>();
    const int lane = threadIdx.x & 31;
    const int64_t pos = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (pos >= hi::plan_count(h.plan, bt)) return;
    const int64_t ch = hi::plan_channel(h.plan, pos, bt);
    const Channel c = channel_of(bt, ch);
    const int64_t tb = h.plan.tile_pref[pos], nt = h.plan.tile_pref[pos + 1] - tb;
    // spans corrected by hi_ufix (processing index >= 1 of channels with a table)
    const int64_t sb = h.plan.span_pref[pos], ns = h.plan.span_pref[pos + 1] - sb;
    const bool fixed = h.span_part != nullptr && ns > 1 && h.hlen[ch] > 0;
    for (int k = lane; k < NACC; k += 32) {
        double v = 0.0;
        for (int64_t i = 0; i < nt; ++i) v += (double)h.partial[(size_t)(tb + i) * NACC + k];
        if (fixed)
            for (int64_t i = 1; i < ns; ++i) v += (double)h.span_part[(size_t)(sb + i) * NACC + k];
        if (k <= MB) {
            if (h.gb && k <= c.N) h.gb[ch * bt.Nstride + k] = (float)v;
        } else {
            const int m = k - MB - 1;
            if (h.ga && m < c.M) h.ga[ch * bt.Mstride + m] = (float)(-v);
        }
    }
    // an empty channel has no adjoint: its state gradient is zero
    if (c.len == 0 && h.gzi && lane < c.M) h.gzi[ch * bt.Mstride + lane] = 0.f;
    if (c.len == 0 && h.gzi && lane + 32 < c.M) h.gzi[ch * bt.Mstride + lane + 32] = 0.f;
}


template <int MB, bool REV>
cudaError_t launch_scan(const HiArgs &h, const Batch &bt, int num_sms, cudaStream_t st) {
    constexpr int TPR = scan_tpr(MB);
    constexpr int NT = MB * TPR;
    auto kern = hi_scan_kernel<MB, TPR, REV>;
    const size_t smem = (size_t)2 * MB * 8 + 32 + (size_t)8 * MB * 4;
    static int occ[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        int o = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, smem);
        if (e != cudaSuccess) return e;
        occ[dev] = o < 1 ? 1 : o;   // resident CTAs per SM
    }
    int want = 0;
    hi_tuning_get(MB, nullptr, &want);
    if (want <= 0) want = hi_scan_chains_default(MB);
    const int per_sm = want < occ[dev] ? want : occ[dev];
    kern<<<(unsigned)(num_sms * per_sm), NT, smem, st>>>(h, bt); note_launch();
    return cudaGetLastError();
}

template <int MB, bool BWD>
cudaError_t launch_e(const HiArgs &h, const Batch &bt, int num_sms, cudaStream_t st) {
    using SM = ESmem<MB>;
    auto kern = hi_e_kernel<MB, BWD>;
    static int occ[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::BYTES);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kChunks, SM::BYTES);
        if (e != cudaSuccess) return e;
        occ[dev] = o < 1 ? 1 : o;
    }
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0 ? 1 : 0; };
    const int st_al = (al(h.states) && bt.Mstride % 4 == 0) ? 1 : 0;
    kern<<<(unsigned)(num_sms * occ[dev]), kChunks, SM::BYTES, st>>>(h, bt, al(h.sig), st_al); note_launch();
    return cudaGetLastError();
}

}  // namespace

template <int MB>
cudaError_t hi_plan(const HiArgs &h, const Batch &bt, cudaStream_t st) {
    hi_plan_kernel<<<1, 1024, 0, st>>>(h.plan, bt); note_launch();
    if (bt.B <= 0) return cudaGetLastError();
    const int64_t blocks = (bt.B + 7) / 8;
    hi_pos_kernel<<<(unsigned)(blocks < 2048 ? blocks : 2048), 256, 0, st>>>(h.plan, bt); note_launch();
    return cudaGetLastError();
}

template <int MB>
cudaError_t hi_jump(const HiArgs &h, const Batch &bt, bool bwd, int num_sms, cudaStream_t st) {
    (void)num_sms;
    constexpr int TPR = scan_tpr(MB);
    const size_t smem = (size_t)(MB * MB + kL + MB + 2 * MB + 2 * kL) * 8 + MB * 4 + 16 + 64;
    auto kern = hi_jump_kernel<MB, TPR>;
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (smem > 48 * 1024 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    // one block per channel position (at most B; blocks past the launch's list exit)
    if (bt.B <= 0) return cudaSuccess;
    kern<<<(unsigned)bt.B, MB * TPR, smem, st>>>(h, bt, bwd ? 1 : 0); note_launch();
    return cudaGetLastError();
}

template <int MB>
cudaError_t hi_scan(const HiArgs &h, const Batch &bt, bool bwd, int num_sms, cudaStream_t st) {
    return bwd ? launch_scan<MB, true>(h, bt, num_sms, st) : launch_scan<MB, false>(h, bt, num_sms, st);
}

template <int MB>
cudaError_t hi_reduce(const HiArgs &h, const Batch &bt, cudaStream_t st) {
    if (bt.B <= 0) return cudaSuccess;
    hi_reduce_kernel<MB><<<(unsigned)((bt.B + 3) / 4), 128, 0, st>>>(h, bt); note_launch();
    return cudaGetLastError();
}

template <int MB>
cudaError_t hi_epass(const HiArgs &h, const Batch &bt, bool bwd, int num_sms, cudaStream_t st) {
    return bwd ? launch_e<MB, true>(h, bt, num_sms, st) : launch_e<MB, false>(h, bt, num_sms, st);
}

template <int MB>
cudaError_t hi_yfix(const HiArgs &h, const Batch &bt, int64_t items_bound, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (int64_t)(sms > 0 ? sms : 1) * 8;
    if (grid > items_bound) grid = items_bound > 0 ? items_bound : 1;
    hi_yfix_kernel<MB><<<(unsigned)grid, 256, 0, st>>>(h, bt); note_launch();
    return cudaGetLastError();
}

template <int MB>
cudaError_t hi_ufix(const HiArgs &h, const Batch &bt, int64_t items_bound, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (int64_t)(sms > 0 ? sms : 1) * 4;
    if (grid > items_bound) grid = items_bound > 0 ? items_bound : 1;
    hi_ufix_kernel<MB><<<(unsigned)grid, 256, 0, st>>>(h, bt); note_launch();
    return cudaGetLastError();
}

template <int MB>
cudaError_t hi_lag(const HiArgs &h, const Batch &bt, int num_sms, cudaStream_t st) {
    using SM = LagSmem<MB>;
    auto kern = hi_lag_kernel<MB>;
    static int occ[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM));
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 256, sizeof(SM));
        if (e != cudaSuccess) return e;
        occ[dev] = o < 1 ? 1 : o;
    }
    kern<<<(unsigned)(num_sms * occ[dev]), 256, sizeof(SM), st>>>(h, bt); note_launch();
    return cudaGetLastError();
}

template cudaError_t hi_plan<DFILT_MB>(const HiArgs &, const Batch &, cudaStream_t);
template cudaError_t hi_jump<DFILT_MB>(const HiArgs &, const Batch &, bool, int, cudaStream_t);
template cudaError_t hi_scan<DFILT_MB>(const HiArgs &, const Batch &, bool, int, cudaStream_t);
template cudaError_t hi_reduce<DFILT_MB>(const HiArgs &, const Batch &, cudaStream_t);
template cudaError_t hi_epass<DFILT_MB>(const HiArgs &, const Batch &, bool, int, cudaStream_t);
template cudaError_t hi_yfix<DFILT_MB>(const HiArgs &, const Batch &, int64_t, cudaStream_t);
template cudaError_t hi_ufix<DFILT_MB>(const HiArgs &, const Batch &, int64_t, cudaStream_t);
template cudaError_t hi_lag<DFILT_MB>(const HiArgs &, const Batch &, int, cudaStream_t);

}  // namespace dfilt
