/*
 * FP64 CPU oracle for the staggered Dirac operator and conjugate gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg use it.  It shares no code with
 * the CUDA path (its own geometry, its own phases, its own algebra).
 *
 * What it computes (Jang, Kim, Lee, "Multi GPU Performance of Conjugate
 * Gradient Solver with Staggered Fermions in Mixed Precision", Lattice 2011):
 *
 *   D chi(x) = sum_mu  s_mu(x)     U_mu(x)        chi(x+mu)
 *                    - s_mu(x-mu)  U_mu(x-mu)^dag chi(x-mu)          (Eq. 5)
 *
 *   with the staggered phase folded into the link, as the paper does in its
 *   gauge-link preconditioning step (Sec. 2, text after Eq. 5):
 *     s_mu(x) = eta_mu(x) * b_mu(x),
 *     eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1})   (mu order x, y, z, t),
 *     b_mu(x)   = -1 if mu = t and x_t = Lt-1, else +1 (antiperiodic in t).
 *   The paper gives neither eta's formula nor the time boundary; this is the
 *   standard reading (MILC/CPS direction order), stated as such.
 *
 *   A = -D^2 + m^2 (Eq. 3), restricted to even sites:
 *     A chi_e = m^2 chi_e - D_eo (D_oe chi_e).
 *
 *   CG exactly as in Fig. 1 (x0 given, r = b - A x0, d = r, alpha =
 *   delta_new / d^dag A d, ...), stopping when delta_new <= tol^2 |b|^2 or
 *   after maxiter iterations; afterwards the true residual b - A x is formed
 *   again and, if it is still above tol |b|, the Fig. 1 loop restarts from it.
 *
 * Layouts (complex128, C order):
 *   links  U[Lt][Lz][Ly][Lx][4][3][3], no phases, no boundary signs;
 *   fields on one parity p: chi[Vh][3], site index i = lex(x) >> 1 over the
 *   sites with (x+y+z+t) % 2 == p, lex(x) = x + Lx*(y + Ly*(z + Lz*t)).
 *
 * Parity pins: see tests/test_oracle_pins.py (free-field closed form,
 * anti-Hermiticity, gauge covariance, dense solves on 2^4 and 4^4).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { ORC_OK = 0, ORC_ERR_DIMS = -1, ORC_ERR_ARG = -2, ORC_ERR_OOM = -3,
       ORC_NOT_CONVERGED = 1, ORC_BREAKDOWN = 2 };

static int check_dims(const int *L)
{
    if (!L) return ORC_ERR_ARG;
    for (int mu = 0; mu < 4; ++mu)
        if (L[mu] < 2 || (L[mu] % 2) != 0) return ORC_ERR_DIMS;
    return ORC_OK;
}

static long volume(const int *L) { return (long)L[0] * L[1] * L[2] * L[3]; }

static long lex(const int *L, const int *c)
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* coordinates of the i-th site of parity p: walk the lexicographic order */
static void coords_of(const int *L, int p, long i, int *c)
{
    /* lex = 2*i or 2*i+1, whichever has parity p */
    long l = 2 * i;
    int t = (int)(l / ((long)L[0] * L[1] * L[2]));
    long rem = l % ((long)L[0] * L[1] * L[2]);
    int z = (int)(rem / ((long)L[0] * L[1]));
    rem %= ((long)L[0] * L[1]);
    int y = (int)(rem / L[0]);
    int x = (int)(rem % L[0]);
    if (((x + y + z + t) & 1) != p) x += 1; /* L[0] even: x+1 stays in range */
    c[0] = x; c[1] = y; c[2] = z; c[3] = t;
}

static int eta(int mu, const int *c)
{
    int s = 0;
    for (int nu = 0; nu < mu; ++nu) s += c[nu];
    return (s & 1) ? -1 : 1;
}

static int bsign(const int *L, int mu, const int *c)
{
    return (mu == 3 && c[3] == L[3] - 1) ? -1 : 1;
}

static const cplx *link_at(const int *L, const cplx *U, const int *c, int mu)
{
    return U + (lex(L, c) * 4 + mu) * 9;
}

/* one output site of D_{p <- 1-p} (Eq. 5) */
static void dslash_site(const int *L, const cplx *U, const cplx *in,
                        const int *c, cplx out[3])
{
    cplx acc[3] = {0, 0, 0};
    for (int mu = 0; mu < 4; ++mu) {
        int cf[4], cb[4];
        memcpy(cf, c, sizeof cf);
        memcpy(cb, c, sizeof cb);
        cf[mu] = (c[mu] + 1) % L[mu];
        cb[mu] = (c[mu] - 1 + L[mu]) % L[mu];

        /* forward hop: s_mu(x) U_mu(x) chi(x+mu) */
        const cplx *uf = link_at(L, U, c, mu);
        const cplx *xf = in + (lex(L, cf) >> 1) * 3;
        double sf = (double)(eta(mu, c) * bsign(L, mu, c));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                acc[a] += sf * uf[a * 3 + b] * xf[b];

        /* backward hop: - s_mu(x-mu) U_mu(x-mu)^dag chi(x-mu) */
        const cplx *ub = link_at(L, U, cb, mu);
        const cplx *xb = in + (lex(L, cb) >> 1) * 3;
        double sb = (double)(eta(mu, cb) * bsign(L, mu, cb));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                acc[a] -= sb * conj(ub[b * 3 + a]) * xb[b];
    }
    out[0] = acc[0]; out[1] = acc[1]; out[2] = acc[2];
}

/* out (parity out_parity, Vh x 3) = D_{out_parity <- other} in */
int orc_dslash(const int *L, const cplx *U, const cplx *in, cplx *out, int out_parity)
{
    int e = check_dims(L);
    if (e) return e;
    if (!U || !in || !out || (out_parity != 0 && out_parity != 1)) return ORC_ERR_ARG;
    long vh = volume(L) / 2;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < vh; ++i) {
        int c[4];
        coords_of(L, out_parity, i, c);
        dslash_site(L, U, in, c, out + i * 3);
    }
    return ORC_OK;
}

/* D_{out_parity <- other} evaluated only at the listed checkerboard sites;
 * out[k] (3 complex) belongs to sites[k]. */
int orc_dslash_sites(const int *L, const cplx *U, const cplx *in, int out_parity,
                     const long *sites, long nsites, cplx *out)
{
    int e = check_dims(L);
    if (e) return e;
    if (!U || !in || !out || !sites || (out_parity != 0 && out_parity != 1)) return ORC_ERR_ARG;
    long vh = volume(L) / 2;
    for (long k = 0; k < nsites; ++k) {
        if (sites[k] < 0 || sites[k] >= vh) return ORC_ERR_ARG;
        int c[4];
        coords_of(L, out_parity, sites[k], c);
        dslash_site(L, U, in, c, out + k * 3);
    }
    return ORC_OK;
}

/* out_e = m^2 in_e - D_eo (D_oe in_e)   (Eq. 3 on even sites) */
static int apply_A_tmp(const int *L, const cplx *U, double mass, const cplx *in,
                       cplx *out, cplx *tmp_odd)
{
    long n = volume(L) / 2 * 3;
    int e = orc_dslash(L, U, in, tmp_odd, 1);
    if (e) return e;
    e = orc_dslash(L, U, tmp_odd, out, 0);
    if (e) return e;
    double m2 = mass * mass;
    for (long k = 0; k < n; ++k) out[k] = m2 * in[k] - out[k];
    return ORC_OK;
}

int orc_apply_A(const int *L, const cplx *U, double mass, const cplx *in, cplx *out)
{
    int e = check_dims(L);
    if (e) return e;
    if (!U || !in || !out) return ORC_ERR_ARG;
    long n = volume(L) / 2 * 3;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
    if (!tmp) return ORC_ERR_OOM;
    e = apply_A_tmp(L, U, mass, in, out, tmp);
    free(tmp);
    return e;
}

static double re_dot(const cplx *a, const cplx *b, long n)
{
    double s = 0.0;
    for (long k = 0; k < n; ++k) s += creal(conj(a[k]) * b[k]);
    return s;
}

/*
 * CG of Fig. 1 on A x = b (even sites).  x holds x0 on entry (zeros for the
 * paper's start) and the solution on exit.  Stops when delta_new <= tol^2
 * |b|^2 (the Fig. 1 test with delta_0 = |b|^2, identical for x0 = 0) or when
 * the total iteration count reaches maxiter.  When the loop stops on the
 * iterated residual, the true residual is recomputed and the Fig. 1 loop
 * restarts from it if |b - A x| > tol |b| (at most `max_restarts` times).
 *
 * info[0] = iterations, info[1] = restarts taken; res[0] = |b - A x| / |b|.
 * Returns ORC_OK, ORC_NOT_CONVERGED or ORC_BREAKDOWN (d^dag A d <= 0).
 */
int orc_cg(const int *L, const cplx *U, double mass, const cplx *b, cplx *x,
           double tol, long maxiter, int max_restarts, long *info, double *res)
{
    int e = check_dims(L);
    if (e) return e;
    if (!U || !b || !x || !info || !res || tol < 0.0 || maxiter < 0) return ORC_ERR_ARG;
    long n = volume(L) / 2 * 3;
    cplx *r = (cplx *)malloc(sizeof(cplx) * n);
    cplx *d = (cplx *)malloc(sizeof(cplx) * n);
    cplx *q = (cplx *)malloc(sizeof(cplx) * n);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
    if (!r || !d || !q || !tmp) { free(r); free(d); free(q); free(tmp); return ORC_ERR_OOM; }

    double bb = re_dot(b, b, n);
    long it = 0;
    int passes = 0, status = ORC_NOT_CONVERGED;
    for (;;) {
        /* r = b - A x, d = r, delta_new = r^dag r */
        apply_A_tmp(L, U, mass, x, q, tmp);
        for (long k = 0; k < n; ++k) { r[k] = b[k] - q[k]; d[k] = r[k]; }
        double delta_new = re_dot(r, r, n);
        if (bb == 0.0 || delta_new <= tol * tol * bb) { status = ORC_OK; break; }
        if (it >= maxiter || passes > max_restarts) break;

        while (it < maxiter && delta_new > tol * tol * bb) {
            apply_A_tmp(L, U, mass, d, q, tmp);
            double dq = re_dot(d, q, n);
            if (!(dq > 0.0)) { status = ORC_BREAKDOWN; goto done; }
            double alpha = delta_new / dq;
            for (long k = 0; k < n; ++k) { x[k] += alpha * d[k]; r[k] -= alpha * q[k]; }
            double delta_old = delta_new;
            delta_new = re_dot(r, r, n);
            double beta = delta_new / delta_old;
            for (long k = 0; k < n; ++k) d[k] = r[k] + beta * d[k];
            ++it;
        }
        ++passes;
    }
done:
    apply_A_tmp(L, U, mass, x, q, tmp);
    for (long k = 0; k < n; ++k) r[k] = b[k] - q[k];
    res[0] = bb > 0.0 ? sqrt(re_dot(r, r, n) / bb) : 0.0;
    info[0] = it;
    info[1] = passes > 0 ? passes - 1 : 0;
    free(r); free(d); free(q); free(tmp);
    return status;
}

/*
 * Mixed-precision CG emulated on the CPU (Fig. 2 with the corrected inner
 * start of Eq. 6 and the reliable / group-wise updates of Sec. 3.2), for the
 * iteration behaviour of the method; not a bitwise model of the GPU (its
 * rounding order differs).  The inner vectors y, r^, d and q are stored in
 * single precision (float complex); A is applied in double to the single-
 * precision d and its result rounded to single; inner products are summed
 * in double.  x, b, the true residual b - A x and the updates are double.
 *
 * Trigger (Sec. 3.2, reading of "Max(|r^y|)"): |r^|^2 < delta_in^2 times the
 * largest |r^|^2 since the last update, or |r^|^2 <= tol^2 |b|^2.  At a
 * trigger: x += y, r = b - A x (double), y = 0, r^ = r (group-wise update);
 * if |r| <= tol |b| the solve ends; else d = r^ + beta d with beta =
 * |r|^2 / (the iterated |r^|^2 before the triggering step) (Eq. 6, d kept).
 * With refine != 0, the plain iterative refinement of Fig. 2 instead: the
 * reference is |r^|^2 at the start of the inner solve, and each inner solve
 * starts again from d = r^.
 *
 * info[0] = inner iterations, info[1] = updates; res[0] = |b - A x| / |b|.
 * Returns ORC_OK, ORC_NOT_CONVERGED or ORC_BREAKDOWN (d^dag A d <= 0).
 *
 * Optional snapshot of the first update that does not end the solve (for
 * the test of Eq. 6; both NULL otherwise): snap_s[0] = the iterated |r^|^2
 * before the triggering step, snap_s[1] = the iterated |r^|^2 after it,
 * snap_s[2] = |r|^2 of the new true residual, snap_s[3] = 1 once taken;
 * snap_v = 4 n values: x after the update, d before it, r^ after it and the
 * new d.  Recording changes none of the arithmetic.
 */
typedef float complex fcplx;

int orc_cg_mixed_snap(const int *L, const cplx *U, double mass, const cplx *b, cplx *x,
                      double tol, double delta_in, long maxiter, int refine, long *info,
                      double *res, double *snap_s, cplx *snap_v)
{
    int e = check_dims(L);
    if (e) return e;
    if (!U || !b || !x || !info || !res || tol < 0.0 || maxiter < 0 ||
        !(delta_in > 0.0 && delta_in < 1.0))
        return ORC_ERR_ARG;
    long n = volume(L) / 2 * 3;
    cplx *rt = (cplx *)malloc(sizeof(cplx) * n);    /* true residual (double) */
    cplx *ad = (cplx *)malloc(sizeof(cplx) * n);    /* A applied in double */
    cplx *wk = (cplx *)malloc(sizeof(cplx) * n);    /* odd intermediate */
    fcplx *ys = (fcplx *)malloc(sizeof(fcplx) * n); /* single-precision vectors */
    fcplx *rs = (fcplx *)malloc(sizeof(fcplx) * n);
    fcplx *ds = (fcplx *)malloc(sizeof(fcplx) * n);
    fcplx *qs = (fcplx *)malloc(sizeof(fcplx) * n);
    if (!rt || !ad || !wk || !ys || !rs || !ds || !qs) {
        free(rt); free(ad); free(wk); free(ys); free(rs); free(ds); free(qs);
        return ORC_ERR_OOM;
    }
    double b2 = re_dot(b, b, n), goal = tol * tol * b2;
    long it = 0, ups = 0;
    int status = ORC_NOT_CONVERGED;

    /* true residual of the start */
    apply_A_tmp(L, U, mass, x, ad, wk);
    for (long k = 0; k < n; ++k) rt[k] = b[k] - ad[k];
    double true2 = re_dot(rt, rt, n);
    if (b2 == 0.0 || true2 <= goal) { status = ORC_OK; goto out; }

    /* inner start: y = 0, r^ = r, d = r^ */
    double rho = 0.0;
    for (long k = 0; k < n; ++k) {
        ys[k] = 0.0f;
        rs[k] = (fcplx)rt[k];
        ds[k] = rs[k];
        rho += creal(conj((cplx)rs[k]) * (cplx)rs[k]);
    }
    double rho_max = rho;
    while (it < maxiter) {
        for (long k = 0; k < n; ++k) wk[k] = (cplx)ds[k];
        apply_A_tmp(L, U, mass, wk, ad, rt);   /* rt serves as the odd scratch here */
        double dAd = 0.0;
        for (long k = 0; k < n; ++k) {
            qs[k] = (fcplx)ad[k];
            dAd += creal(conj((cplx)ds[k]) * (cplx)qs[k]);
        }
        if (!(dAd > 0.0)) { status = ORC_BREAKDOWN; break; }
        double step = rho / dAd;
        double rho_prev = rho;
        rho = 0.0;
        for (long k = 0; k < n; ++k) {
            ys[k] = (fcplx)((cplx)ys[k] + step * (cplx)ds[k]);
            rs[k] = (fcplx)((cplx)rs[k] - step * (cplx)qs[k]);
            rho += creal(conj((cplx)rs[k]) * (cplx)rs[k]);
        }
        ++it;
        if (!refine && rho > rho_max) rho_max = rho;
        double mult;
        if (rho < delta_in * delta_in * rho_max || rho <= goal) {
            /* reliable update (x += y) and group-wise update (r^ = b - A x) */
            for (long k = 0; k < n; ++k) x[k] += (cplx)ys[k];
            apply_A_tmp(L, U, mass, x, ad, wk);
            for (long k = 0; k < n; ++k) rt[k] = b[k] - ad[k];
            true2 = re_dot(rt, rt, n);
            ++ups;
            if (true2 <= goal) { status = ORC_OK; break; }
            for (long k = 0; k < n; ++k) { ys[k] = 0.0f; rs[k] = (fcplx)rt[k]; }
            const int snap = snap_s && snap_v && snap_s[3] == 0.0;
            if (snap) {
                snap_s[0] = rho_prev;
                snap_s[1] = rho;
                snap_s[2] = true2;
                snap_s[3] = 1.0;
                for (long k = 0; k < n; ++k) {
                    snap_v[k] = x[k];
                    snap_v[n + k] = (cplx)ds[k];
                    snap_v[2 * n + k] = (cplx)rs[k];
                }
            }
            mult = refine ? 0.0 : true2 / rho_prev;   /* Eq. 6; Fig. 2 restarts d */
            for (long k = 0; k < n; ++k) ds[k] = (fcplx)((cplx)rs[k] + mult * (cplx)ds[k]);
            if (snap)
                for (long k = 0; k < n; ++k) snap_v[3 * n + k] = (cplx)ds[k];
            rho = 0.0;
            for (long k = 0; k < n; ++k) rho += creal(conj((cplx)rs[k]) * (cplx)rs[k]);
            rho_max = rho;
        } else {
            mult = rho / rho_prev;
            for (long k = 0; k < n; ++k) ds[k] = (fcplx)((cplx)rs[k] + mult * (cplx)ds[k]);
        }
    }
out:
    apply_A_tmp(L, U, mass, x, ad, wk);
    for (long k = 0; k < n; ++k) rt[k] = b[k] - ad[k];
    res[0] = b2 > 0.0 ? sqrt(re_dot(rt, rt, n) / b2) : 0.0;
    info[0] = it;
    info[1] = ups;
    free(rt); free(ad); free(wk); free(ys); free(rs); free(ds); free(qs);
    return status;
}

int orc_cg_mixed(const int *L, const cplx *U, double mass, const cplx *b, cplx *x,
                 double tol, double delta_in, long maxiter, int refine, long *info, double *res)
{
    return orc_cg_mixed_snap(L, U, mass, b, x, tol, delta_in, maxiter, refine, info, res,
                             NULL, NULL);
}

int orc_version(void) { return 1; }
