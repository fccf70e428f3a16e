/*
 * FP64 CPU oracle for batched direct-form IIR filters and their closed-form
 * gradients.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library; the product path
 * (the CUDA library and its Python binding) never does, and shares no code,
 * header, table or constant with it.
 *
 * Notation (paper, Eq. rtf and Sec. 2): per channel
 *     H(z) = (b_0 + b_1 z^-1 + ... + b_N z^-N) / (1 + a_1 z^-1 + ... + a_M z^-M)
 * with b zero-padded to order M (the paper pads the shorter polynomial, Sec. 2).
 * The coefficient array `a` holds a_1..a_M (a_0 = 1 is implicit), so a[k-1] is a_k.
 *
 * Initial state zi[0..M) follows the transposed direct form II (TDF-II, the form
 * the paper names for SciPy/MATLAB in Sec. 2): zi is the TDF-II state vector at
 * n = 0.  Equivalently zi[k] is added to the all-pole input at time k (k < M).
 *
 * Every function here is the plain definition, looped in the paper's order, in
 * double precision.  Nothing is blocked, fused or reordered.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* b_k with the zero padding of Sec. 2 (k > N gives 0). */
static double bcoef(const double *b, int N, int k) { return k <= N ? b[k] : 0.0; }

/*
 * Forward, TDF-II state recursion (Sec. 2: state-space form with A replaced by
 * its transpose and B, C swapped, i.e. Eqs. ss_recursion/ss_output for TDF):
 *     y[n]   = b_0 x[n] + s_0
 *     s_k   <- s_{k+1} + b_{k+1} x[n] - a_{k+1} y[n]     (k = 0..M-1, s_M = 0)
 * starting from s = zi.
 */
static void fwd_tdf2(const double *x, const double *b, const double *a, const double *zi,
                     double *y, int64_t T, int N, int M, double *s)
{
    for (int k = 0; k < M; ++k) s[k] = zi ? zi[k] : 0.0;
    for (int64_t n = 0; n < T; ++n) {
        const double xn = x[n];
        const double yn = b[0] * xn + s[0];
        for (int k = 0; k < M; ++k) {
            const double nxt = (k + 1 < M) ? s[k + 1] : 0.0;
            s[k] = nxt + bcoef(b, N, k + 1) * xn - a[k] * yn;
        }
        y[n] = yn;
    }
}

/*
 * Forward, the same filter written as the difference equation of Eq. rtf with
 * the initial state injected into the recursion input:
 *     w[n] = sum_{k=0..N} b_k x[n-k] + zi[n] [n < M]
 *     y[n] = w[n] - sum_{k=1..M} a_k y[n-k]
 * (x, y are zero at negative times).  A second formulation used to cross-check
 * the state recursion above.
 */
static void fwd_injection(const double *x, const double *b, const double *a, const double *zi,
                          double *y, int64_t T, int N, int M)
{
    for (int64_t n = 0; n < T; ++n) {
        double w = 0.0;
        for (int k = 0; k <= N; ++k)
            if (n - k >= 0) w += b[k] * x[n - k];
        if (zi && n < M) w += zi[n];
        double acc = w;
        for (int k = 1; k <= M; ++k)
            if (n - k >= 0) acc -= a[k - 1] * y[n - k];
        y[n] = acc;
    }
}

/*
 * Backward: the reverse-time adjoint recursion (Eqs. dLdz, dLdx, dLdvBA and the
 * boundary condition of App. A, dL/dz(N-1) = 0), in scalar difference form:
 *     u[n]       = g[n] - sum_{k=1..M} a_k u[n+k],        u[n >= T] = 0
 *     grad_x[n]  = sum_{k=0..N} b_k u[n+k]
 *     grad_b[k]  = sum_{n=k..T-1} u[n] x[n-k]             (k = 0..N)
 *     grad_a[k]  = -sum_{n=k..T-1} u[n] y[n-k]            (k = 1..M)
 *     grad_zi[k] = u[k]                                   (k = 0..M-1; 0 if k >= T)
 * u is the gradient with respect to the all-pole input; grad_zi is the gradient
 * with respect to the initial state (App. A, dL/dv(0)).
 * Any output pointer may be NULL (not requested).  u is caller scratch [T].
 */
static void bwd_channel(const double *g, const double *x, const double *y,
                        const double *b, const double *a,
                        double *gx, double *gb, double *ga, double *gzi,
                        int64_t T, int N, int M, double *u)
{
    for (int64_t n = T - 1; n >= 0; --n) {
        double acc = g[n];
        for (int k = 1; k <= M; ++k)
            if (n + k < T) acc -= a[k - 1] * u[n + k];
        u[n] = acc;
    }
    if (gx)
        for (int64_t n = 0; n < T; ++n) {
            double acc = 0.0;
            for (int k = 0; k <= N; ++k)
                if (n + k < T) acc += b[k] * u[n + k];
            gx[n] = acc;
        }
    if (gb)
        for (int k = 0; k <= N; ++k) {
            double acc = 0.0;
            for (int64_t n = k; n < T; ++n) acc += u[n] * x[n - k];
            gb[k] = acc;
        }
    if (ga)
        for (int k = 1; k <= M; ++k) {
            double acc = 0.0;
            for (int64_t n = k; n < T; ++n) acc += u[n] * y[n - k];
            ga[k - 1] = -acc;
        }
    if (gzi)
        for (int k = 0; k < M; ++k) gzi[k] = (k < T) ? u[k] : 0.0;
}

static int pick_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * Ragged batch drivers.  Channel i owns samples [offs[i], offs[i+1]) of the packed
 * signal arrays, has orders Ms[i], Ns[i] (1 <= Ms[i] <= Mmax, 0 <= Ns[i] <= Ms[i]) and
 * coefficient rows b + i*(Nmax+1), a + i*Mmax, zi + i*Mmax (zi may be NULL).
 * `form` selects the forward formulation: 0 = TDF-II state, 1 = injection.
 * Returns 0, or -1 on an allocation failure.
 */
int oracle_forward_ragged(const double *x, const int64_t *offs, const int *Ms, const int *Ns,
                          const double *b, const double *a, const double *zi, double *y,
                          int64_t B, int Nmax, int Mmax, int form, int nthreads)
{
    int fail = 0;
    const int nt = pick_threads(nthreads);
#pragma omp parallel num_threads(nt)
    {
        double *s = (double *)malloc(sizeof(double) * (size_t)(Mmax > 0 ? Mmax : 1));
        if (!s) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < B; ++i) {
            if (!s) continue;
            const int64_t o = offs[i], T = offs[i + 1] - offs[i];
            const double *zii = zi ? zi + i * Mmax : NULL;
            if (form == 0)
                fwd_tdf2(x + o, b + i * (Nmax + 1), a + i * Mmax, zii, y + o, T, Ns[i], Ms[i], s);
            else
                fwd_injection(x + o, b + i * (Nmax + 1), a + i * Mmax, zii, y + o, T, Ns[i], Ms[i]);
        }
        free(s);
    }
    return fail ? -1 : 0;
}

int oracle_backward_ragged(const double *g, const double *x, const double *y,
                           const int64_t *offs, const int *Ms, const int *Ns,
                           const double *b, const double *a,
                           double *gx, double *gb, double *ga, double *gzi,
                           int64_t B, int Nmax, int Mmax, int nthreads)
{
    int fail = 0;
    int64_t Tmax = 0;
    for (int64_t i = 0; i < B; ++i)
        if (offs[i + 1] - offs[i] > Tmax) Tmax = offs[i + 1] - offs[i];
    const int nt = pick_threads(nthreads);
#pragma omp parallel num_threads(nt)
    {
        double *u = (double *)malloc(sizeof(double) * (size_t)(Tmax > 0 ? Tmax : 1));
        if (!u) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < B; ++i) {
            if (!u) continue;
            const int64_t o = offs[i], T = offs[i + 1] - offs[i];
            bwd_channel(g + o, x + o, y + o, b + i * (Nmax + 1), a + i * Mmax,
                        gx ? gx + o : NULL, gb ? gb + i * (Nmax + 1) : NULL,
                        ga ? ga + i * Mmax : NULL, gzi ? gzi + i * Mmax : NULL,
                        T, Ns[i], Ms[i], u);
        }
        free(u);
    }
    return fail ? -1 : 0;
}

/*
 * Forward mode (JVP): the directional derivative of the forward along tangents
 * (dx, db, da, dzi), for the forward-mode derivative the paper notes can be derived
 * the same way as the reverse mode (Sec. 5).  Written as the TDF-II state recursion
 * of fwd_tdf2 carried together with its derivative (dual numbers): every primal
 * assignment is followed by its product-rule derivative,
 *     y[n]   = b_0 x[n] + s_0
 *     dy[n]  = db_0 x[n] + b_0 dx[n] + ds_0
 *     s_k   <- s_{k+1} + b_{k+1} x[n] - a_{k+1} y[n]
 *     ds_k  <- ds_{k+1} + db_{k+1} x[n] + b_{k+1} dx[n] - da_{k+1} y[n] - a_{k+1} dy[n]
 * starting from s = zi, ds = dzi.  A NULL tangent is zero.  s, ds are caller
 * scratch [M].
 */
static void jvp_tdf2(const double *x, const double *b, const double *a, const double *zi,
                     const double *dx, const double *db, const double *da, const double *dzi,
                     double *y, double *dy, int64_t T, int N, int M, double *s, double *ds)
{
    for (int k = 0; k < M; ++k) {
        s[k] = zi ? zi[k] : 0.0;
        ds[k] = dzi ? dzi[k] : 0.0;
    }
    for (int64_t n = 0; n < T; ++n) {
        const double xn = x[n];
        const double dxn = dx ? dx[n] : 0.0;
        const double yn = xn * b[0] + s[0];
        double dyn = b[0] * dxn + ds[0];
        if (db) dyn += db[0] * xn;
        for (int k = 0; k < M; ++k) {
            const double nxt = (k + 1 < M) ? s[k + 1] : 0.0;
            const double dnxt = (k + 1 < M) ? ds[k + 1] : 0.0;
            s[k] = nxt + xn * bcoef(b, N, k + 1) - yn * a[k];
            double d = dnxt + bcoef(b, N, k + 1) * dxn - a[k] * dyn;
            if (db) d += bcoef(db, N, k + 1) * xn;
            if (da) d -= da[k] * yn;
            ds[k] = d;
        }
        y[n] = yn;
        dy[n] = dyn;
    }
}

/*
 * Fixed-shape batch driver of jvp_tdf2: channel i owns x + i*T (likewise dx, y, dy)
 * and coefficient rows b + i*(N+1), a + i*M, zi + i*M (and the tangents').  Any of
 * zi, dx, db, da, dzi may be NULL.  Returns 0, or -1 on an allocation failure.
 */
int oracle_jvp(const double *x, const double *b, const double *a, const double *zi,
               const double *dx, const double *db, const double *da, const double *dzi,
               double *y, double *dy, int64_t B, int64_t T, int N, int M, int nthreads)
{
    int fail = 0;
    const int nt = pick_threads(nthreads);
#pragma omp parallel num_threads(nt)
    {
        double *s = (double *)malloc(sizeof(double) * 2 * (size_t)(M > 0 ? M : 1));
        if (!s) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < B; ++i) {
            if (!s) continue;
            const int64_t o = i * T;
            jvp_tdf2(x + o, b + i * (N + 1), a + i * M, zi ? zi + i * M : NULL,
                     dx ? dx + o : NULL, db ? db + i * (N + 1) : NULL, da ? da + i * M : NULL,
                     dzi ? dzi + i * M : NULL, y + o, dy + o, T, N, M, s, s + (M > 0 ? M : 1));
        }
        free(s);
    }
    return fail ? -1 : 0;
}

/*
 * Direct-form initial conditions (the DF-I state: past inputs x[-1..-N] and past
 * outputs y[-1..-M], the convention of SciPy's lfiltic and MATLAB's filtic), the
 * counterpart of the TDF-II state that Sec. 2 pairs with the direct form.  Forward:
 * the difference equation of Eq. rtf over the signals extended into negative time,
 *     xe(i) = x[i] (i >= 0), xpast[-i-1] (i < 0);   ye likewise with ypast
 *     y[n]  = sum_{k=0..N} b_k xe(n-k) - sum_{k=1..M} a_k ye(n-k)
 * Backward: with the adjoint u of bwd_channel (same recursion), the gradients of the
 * same equation with respect to every quantity in it:
 *     grad_b[k]       = sum_{n>=0} u[n] xe(n-k)        (past inputs included)
 *     grad_a[k]       = -sum_{n>=0} u[n] ye(n-k)       (past outputs included)
 *     grad_xpast[j-1] = sum_{k=j..N} b_k u[k-j]        (x[-j] enters y[k-j] via b_k)
 *     grad_ypast[j-1] = -sum_{k=j..M} a_k u[k-j]
 * (u[n] = 0 for n >= T).  grad_x is unchanged.  xpast may be NULL when N = 0.
 */
static double xe_at(const double *x, const double *xp, int64_t i)
{
    return i >= 0 ? x[i] : (xp ? xp[-i - 1] : 0.0);
}

static void fwd_df1_past(const double *x, const double *b, const double *a, const double *xp,
                         const double *yp, double *y, int64_t T, int N, int M)
{
    for (int64_t n = 0; n < T; ++n) {
        double acc = 0.0;
        for (int k = 0; k <= N; ++k) acc += b[k] * xe_at(x, xp, n - k);
        for (int k = 1; k <= M; ++k) acc -= a[k - 1] * (n - k >= 0 ? y[n - k] : yp[k - n - 1]);
        y[n] = acc;
    }
}

static void bwd_df1_past(const double *g, const double *x, const double *y, const double *b,
                         const double *a, const double *xp, const double *yp, double *gx,
                         double *gb, double *ga, double *gxp, double *gyp, int64_t T, int N,
                         int M, double *u)
{
    bwd_channel(g, x, y, b, a, gx, NULL, NULL, NULL, T, N, M, u);
    for (int k = 0; k <= N; ++k) {
        double sum = 0.0;
        for (int64_t n = 0; n < T; ++n) sum += u[n] * xe_at(x, xp, n - k);
        gb[k] = sum;
    }
    for (int k = 1; k <= M; ++k) {
        double sum = 0.0;
        for (int64_t n = 0; n < T; ++n) sum += u[n] * (n - k >= 0 ? y[n - k] : yp[k - n - 1]);
        ga[k - 1] = -sum;
    }
    for (int j = 1; j <= N; ++j) {
        double sum = 0.0;
        for (int k = j; k <= N; ++k)
            if (k - j < T) sum += b[k] * u[k - j];
        gxp[j - 1] = sum;
    }
    for (int j = 1; j <= M; ++j) {
        double sum = 0.0;
        for (int k = j; k <= M; ++k)
            if (k - j < T) sum += a[k - 1] * u[k - j];
        gyp[j - 1] = -sum;
    }
}

/*
 * Fixed-shape drivers: x, y, g [B,T]; b [B,N+1]; a [B,M]; xpast [B,N] (NULL if N = 0);
 * ypast [B,M].  Returns 0, or -1 on an allocation failure.
 */
int oracle_forward_df1(const double *x, const double *b, const double *a, const double *xp,
                       const double *yp, double *y, int64_t B, int64_t T, int N, int M,
                       int nthreads)
{
    const int nt = pick_threads(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
    for (int64_t i = 0; i < B; ++i)
        fwd_df1_past(x + i * T, b + i * (N + 1), a + i * M, (xp && N > 0) ? xp + i * N : NULL,
                     yp + i * M, y + i * T, T, N, M);
    return 0;
}

int oracle_backward_df1(const double *g, const double *x, const double *y, const double *b,
                        const double *a, const double *xp, const double *yp, double *gx,
                        double *gb, double *ga, double *gxp, double *gyp, int64_t B, int64_t T,
                        int N, int M, int nthreads)
{
    int fail = 0;
    const int nt = pick_threads(nthreads);
#pragma omp parallel num_threads(nt)
    {
        double *u = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
        if (!u) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < B; ++i) {
            if (!u) continue;
            bwd_df1_past(g + i * T, x + i * T, y + i * T, b + i * (N + 1), a + i * M,
                         (xp && N > 0) ? xp + i * N : NULL, yp + i * M, gx + i * T,
                         gb + i * (N + 1), ga + i * M, gxp ? gxp + i * (N > 0 ? N : 0) : NULL,
                         gyp + i * M, T, N, M, u);
        }
        free(u);
    }
    return fail ? -1 : 0;
}

/*
 * Parameter-varying direct form (Sec. 5 notes the derivation extends to it): the
 * coefficients of output sample n are b[n][0..N], a[n][0..M-1] (a[n][k-1] = a_k at n),
 *     y[n] = sum_{k=0..N} b[n][k] x[n-k] - sum_{k=1..M} a[n][k-1] y[n-k],
 * x[n < 0] = 0, y[-1-j] = ypast[j] (NULL = zero).  The backward follows the same steps
 * as the fixed-coefficient one with each coefficient taken at the output it produced:
 *     u[n] = g[n] - sum_{k=1..M} a[n+k][k-1] u[n+k]          (u[n >= T] = 0)
 *     grad_x[n] = sum_{k=0..N} b[n+k][k] u[n+k]
 *     grad_b[n][k] = u[n] x[n-k],   grad_a[n][k-1] = -u[n] y[n-k]   (y past: ypast)
 *     grad_ypast[j] = -sum_{k=j+1..M} a[k-1-j][k-1] u[k-1-j]
 */
static void fwd_tv(const double *x, const double *b, const double *a, const double *yp,
                   double *y, int64_t T, int N, int M)
{
    for (int64_t n = 0; n < T; ++n) {
        double acc = 0.0;
        for (int k = 0; k <= N; ++k)
            if (n - k >= 0) acc += b[n * (N + 1) + k] * x[n - k];
        for (int k = 1; k <= M; ++k) {
            const double yk = n - k >= 0 ? y[n - k] : (yp ? yp[k - n - 1] : 0.0);
            acc -= a[n * M + k - 1] * yk;
        }
        y[n] = acc;
    }
}

static void bwd_tv(const double *g, const double *x, const double *y, const double *b,
                   const double *a, const double *yp, double *gx, double *gb, double *ga,
                   double *gyp, int64_t T, int N, int M, double *u)
{
    for (int64_t n = T - 1; n >= 0; --n) {
        double acc = g[n];
        for (int k = 1; k <= M; ++k)
            if (n + k < T) acc -= a[(n + k) * M + k - 1] * u[n + k];
        u[n] = acc;
    }
    for (int64_t n = 0; n < T; ++n) {
        double acc = 0.0;
        for (int k = 0; k <= N; ++k)
            if (n + k < T) acc += b[(n + k) * (N + 1) + k] * u[n + k];
        gx[n] = acc;
        for (int k = 0; k <= N; ++k) gb[n * (N + 1) + k] = n - k >= 0 ? u[n] * x[n - k] : 0.0;
        for (int k = 1; k <= M; ++k) {
            const double yk = n - k >= 0 ? y[n - k] : (yp ? yp[k - n - 1] : 0.0);
            ga[n * M + k - 1] = -u[n] * yk;
        }
    }
    if (gyp) {
        for (int j = 0; j < M; ++j) {
            double acc = 0.0;
            for (int k = j + 1; k <= M; ++k)
                if (k - 1 - j < T) acc += a[(k - 1 - j) * M + k - 1] * u[k - 1 - j];
            gyp[j] = -acc;
        }
    }
}

/* x, y, g [B,T]; b [B,T,N+1]; a [B,T,M]; ypast [B,M] or NULL.  Returns 0 or -1. */
int oracle_forward_tv(const double *x, const double *b, const double *a, const double *yp,
                      double *y, int64_t B, int64_t T, int N, int M, int nthreads)
{
    const int nt = pick_threads(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
    for (int64_t i = 0; i < B; ++i)
        fwd_tv(x + i * T, b + i * T * (N + 1), a + i * T * M, yp ? yp + i * M : NULL, y + i * T,
               T, N, M);
    return 0;
}

int oracle_backward_tv(const double *g, const double *x, const double *y, const double *b,
                       const double *a, const double *yp, double *gx, double *gb, double *ga,
                       double *gyp, int64_t B, int64_t T, int N, int M, int nthreads)
{
    int fail = 0;
    const int nt = pick_threads(nthreads);
#pragma omp parallel num_threads(nt)
    {
        double *u = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
        if (!u) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < B; ++i) {
            if (!u) continue;
            bwd_tv(g + i * T, x + i * T, y + i * T, b + i * T * (N + 1), a + i * T * M,
                   yp ? yp + i * M : NULL, gx + i * T, gb + i * T * (N + 1), ga + i * T * M,
                   gyp ? gyp + i * M : NULL, T, N, M, u);
        }
        free(u);
    }
    return fail ? -1 : 0;
}

/* Threads an OpenMP region actually gets (for reporting the CPU baseline). */
int oracle_max_threads(void) { return pick_threads(0); }
