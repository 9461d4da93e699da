/*
 * nmodl_oracle.c -- plain FP64 CPU oracle of the NMODL mechanism hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Every routine is the definition written out: scalar loops per instance in
 * double precision, libm exp/expm1/pow, a dense LU with partial pivoting.
 * No blocking, fusion or reordering.  Build with -O2 -ffp-contract=off so
 * that no multiply-add is fused behind the reader's back.
 *
 * What the paper fixes, and the readings taken where it is silent:
 *  - Section 1 / Fig. 1: each mechanism has a state update (nrn_state) and
 *    a current update (nrn_cur) kernel, called once per time step.
 *  - Section 3 (BREAKPOINT bullet) and Section 5.2 (CONDUCTANCE): the
 *    current of an ohmic channel is i = g (v - e) and its derivative
 *    dI/dv = g is taken analytically.  Reading: the current update
 *    scatter-adds rhs[node] -= i and d[node] += g (NEURON convention).
 *  - Section 5.1 / 5.2 (cnexp): a linear, independent gate ODE
 *    m' = (minf - m)/mtau is integrated exactly with minf, mtau held
 *    constant over the step:  m += (1 - exp(-dt/mtau)) (minf - m).
 *  - Section 5.1 / 5.2 (KINETIC -> DERIVATIVE, implicit Euler, sparse and
 *    derivimplicit) and Section 5.3 (PartialPivLU, Newton with the exact
 *    Jacobian): a mass-action scheme becomes x' = A(v) x; one implicit
 *    Euler step solves F(y) = y - x - dt A y = 0 by Newton with J = I - dt A.
 *  - Readings (not in the paper): Hodgkin-Huxley 1952 rates in the modern
 *    convention; the step order zero -> cur (mechanism list order,
 *    ascending instance) -> d += 1e-3 cm/dt -> v += rhs/d -> state; the
 *    3x3 lattice topology of the 9-state scheme; vtrap evaluated through
 *    expm1 with a 3-term Taylor branch for |x/y| < 1e-6.
 *  - Section 3 (USEION and the ion dependencies it declares): ion currents
 *    are written per node (ina, ik, ica) by the current update of every
 *    step, before the state updates that read them (calcium accumulation
 *    reads ica).  Readings: the 3-state triangle scheme (Section 5.2
 *    "sparse" for <= 3 equations) and the 2-state calcium buffer of the
 *    derivimplicit kind (Section 5.3 small-matrix Newton).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TYPE_HH 1
#define ORC_TYPE_CNEXP 2
#define ORC_TYPE_KIN9 3
#define ORC_TYPE_CACUM 4
#define ORC_TYPE_KIN3 5
#define ORC_NION 4 /* 0 nonspecific, 1 na, 2 k, 3 ca */

/* ---------------------------------------------------------------- rates */

/* vtrap(x, y) = x / (exp(x/y) - 1), the HH "linoid" rate shape; continuous
 * at x = 0 where it equals y.  expm1 evaluates the same function without the
 * cancellation of exp(x/y) - 1 near zero. */
double orc_vtrap(double x, double y)
{
    double u = x / y;
    if (fabs(u) < 1e-6)
        return y * (1.0 - u / 2.0 + u * u / 12.0);
    return x / expm1(u);
}

/* Hodgkin-Huxley (1952) gate rates, modern sign convention, in 1/ms.
 * minf = alpha/(alpha+beta), mtau = 1/(q10 (alpha+beta)) (rates procedure
 * of the HH example channel; Section 3 inlining / localiser discussion). */
void orc_hh_rates(const double *p, double v, double minf[3], double mtau[3])
{
    double celsius = p[6];
    double q10 = pow(3.0, (celsius - 6.3) / 10.0);
    double a, b;
    /* m */
    a = 0.1 * orc_vtrap(-(v + 40.0), 10.0);
    b = 4.0 * exp(-(v + 65.0) / 18.0);
    minf[0] = a / (a + b);
    mtau[0] = 1.0 / (q10 * (a + b));
    /* h */
    a = 0.07 * exp(-(v + 65.0) / 20.0);
    b = 1.0 / (1.0 + exp(-(v + 35.0) / 10.0));
    minf[1] = a / (a + b);
    mtau[1] = 1.0 / (q10 * (a + b));
    /* n */
    a = 0.01 * orc_vtrap(-(v + 55.0), 10.0);
    b = 0.125 * exp(-(v + 65.0) / 80.0);
    minf[2] = a / (a + b);
    mtau[2] = 1.0 / (q10 * (a + b));
}

/* Generic rate shapes of the cnexp channel family, u = (v - vh)/k. */
double orc_rate(int form, double A, double vh, double k, double v)
{
    double u = (v - vh) / k;
    switch (form) {
    case 0: /* EXP */
        return A * exp(u);
    case 1: /* SIGMOID */
        return A / (1.0 + exp(-u));
    case 2: /* LINOID: A u / (1 - exp(-u)) = A vtrap(-u, 1) */
        if (fabs(u) < 1e-6)
            return A * (1.0 + u / 2.0 + u * u / 12.0);
        return A * u / (-expm1(-u));
    default:
        return NAN;
    }
}

/* minf and mtau of gate g of a CNEXP block at voltage v. */
void orc_cnexp_rates(const double *p, int g, double v, double *minf, double *mtau)
{
    const double *q = p + 6 + 9 * g;
    double phi = pow(p[3], (p[4] - p[5]) / 10.0);
    double a = orc_rate((int)q[1], q[2], q[3], q[4], v);
    double b = orc_rate((int)q[5], q[6], q[7], q[8], v);
    *minf = a / (a + b);
    *mtau = 1.0 / (phi * (a + b));
}

static int n_gates_of(int type, const double *p)
{
    if (type == ORC_TYPE_HH) return 3;
    if (type == ORC_TYPE_CNEXP) return (int)p[0];
    if (type == ORC_TYPE_KIN9) return 9;
    if (type == ORC_TYPE_CACUM) return 2;
    if (type == ORC_TYPE_KIN3) return 3;
    return -1;
}

/* -------------------------------------------------------- init / state */

/* Gates start at their steady state minf(v) (INITIAL block convention). */
static void cnexp_like_init(int type, int64_t n, const int32_t *ni,
                            const double *v, const double *p, double *s)
{
    int ng = n_gates_of(type, p);
    for (int64_t i = 0; i < n; ++i) {
        double vv = v[ni[i]];
        for (int g = 0; g < ng; ++g) {
            double minf, mtau;
            if (type == ORC_TYPE_HH) {
                double mi[3], mt[3];
                orc_hh_rates(p, vv, mi, mt);
                minf = mi[g];
                (void)mt;
            } else {
                orc_cnexp_rates(p, g, vv, &minf, &mtau);
            }
            s[g * n + i] = minf;
        }
    }
}

/* Integration factor of the gate update over x = dt/mtau: 1 - exp(-x)
 * (cnexp, Section 5.2), or with exp(-x) replaced by its (1,1) Pade
 * approximant (1 - x/2)/(1 + x/2) (the optional cheaper form the paper
 * names in Section 5.2). */
int orc_pade_mode = 0;

double orc_cnexp_factor(double x)
{
    if (orc_pade_mode)
        return 1.0 - (1.0 - x / 2.0) / (1.0 + x / 2.0);
    return 1.0 - exp(-x);
}

/* cnexp (Section 5.2): exact solution of m' = (minf - m)/mtau over dt with
 * minf, mtau frozen at the new voltage. */
static void cnexp_like_state(int type, int64_t n, const int32_t *ni,
                             const double *v, const double *p, double dt,
                             double *s)
{
    int ng = n_gates_of(type, p);
    for (int64_t i = 0; i < n; ++i) {
        double vv = v[ni[i]];
        double minf[3], mtau[3];
        if (type == ORC_TYPE_HH) {
            orc_hh_rates(p, vv, minf, mtau);
        } else {
            for (int g = 0; g < ng; ++g)
                orc_cnexp_rates(p, g, vv, &minf[g], &mtau[g]);
        }
        for (int g = 0; g < ng; ++g) {
            double m = s[g * n + i];
            s[g * n + i] = m + orc_cnexp_factor(dt / mtau[g]) * (minf[g] - m);
        }
    }
}

/* -------------------------------------------------------------- currents */

/* Per-instance current i [mA/cm2] and conductance g = dI/dv [S/cm2]. */
static void instance_current(int type, int64_t n, int64_t i, double vv,
                             const double *p, const double *s,
                             double *cur, double *cond)
{
    if (type == ORC_TYPE_HH) {
        double m = s[i], h = s[n + i], nn = s[2 * n + i];
        double gna = p[0] * m * m * m * h;
        double gk = p[1] * nn * nn * nn * nn;
        double gl = p[2];
        *cur = gna * (vv - p[3]) + gk * (vv - p[4]) + gl * (vv - p[5]);
        *cond = gna + gk + gl;
    } else if (type == ORC_TYPE_CNEXP) {
        int ng = (int)p[0];
        double g = p[1];
        for (int k = 0; k < ng; ++k) {
            int pw = (int)p[6 + 9 * k];
            double x = s[k * n + i];
            for (int e = 0; e < pw; ++e)
                g *= x;
        }
        *cur = g * (vv - p[2]);
        *cond = g;
    } else if (type == ORC_TYPE_CACUM) { /* no membrane current */
        *cur = 0.0;
        *cond = 0.0;
    } else { /* KIN9, KIN3: open-state occupancy */
        int op = (int)p[2];
        double g = p[0] * s[op * n + i];
        *cur = g * (vv - p[1]);
        *cond = g;
    }
}

/* Ion currents of an instance (USEION WRITE): HH writes ina (gna term) and
 * ik (gk term); a CNEXP, KIN9 or KIN3 mechanism writes its whole current to the
 * ion it is tagged with (0 = nonspecific, not written). */
static void instance_ion_currents(int type, int ion, int64_t n, int64_t i, double vv,
                                  const double *p, const double *s, double *ic)
{
    for (int k = 0; k < ORC_NION; ++k)
        ic[k] = 0.0;
    if (type == ORC_TYPE_HH) {
        double m = s[i], h = s[n + i], nn = s[2 * n + i];
        ic[1] = p[0] * m * m * m * h * (vv - p[3]);
        ic[2] = p[1] * nn * nn * nn * nn * (vv - p[4]);
    } else if (ion > 0 && type != ORC_TYPE_CACUM) {
        double c, g;
        instance_current(type, n, i, vv, p, s, &c, &g);
        ic[ion] = c;
    }
}

/* ion_i[k][node] += ion current k of every instance (k = 1..3; arrays may
 * be NULL). */
void orc_mech_ion_cur(int type, int ion, int64_t n, const int32_t *ni, const double *v,
                      const double *p, const double *s, double *const *ion_i)
{
    for (int64_t i = 0; i < n; ++i) {
        double ic[ORC_NION];
        instance_ion_currents(type, ion, n, i, v[ni[i]], p, s, ic);
        for (int k = 1; k < ORC_NION; ++k)
            if (ion_i[k])
                ion_i[k][ni[i]] += ic[k];
    }
}

/* Current update: rhs[node] -= i, d[node] += g, ascending instance order. */
void orc_mech_cur(int type, int64_t n, const int32_t *ni, const double *v,
                  const double *p, const double *s, double *rhs, double *d)
{
    for (int64_t i = 0; i < n; ++i) {
        double c, g;
        instance_current(type, n, i, v[ni[i]], p, s, &c, &g);
        rhs[ni[i]] -= c;
        d[ni[i]] += g;
    }
}

/* Per-instance current and conductance, for instance-level checks. */
void orc_mech_currents(int type, int64_t n, const int32_t *ni, const double *v,
                       const double *p, const double *s, double *cur, double *cond)
{
    for (int64_t i = 0; i < n; ++i)
        instance_current(type, n, i, v[ni[i]], p, s, &cur[i], &cond[i]);
}

/* ------------------------------------------------------------ kinetic 9 */

/* Generator matrix of the 3x3 lattice scheme, row-major A[r*9+c]:
 * A[j][i] = rate i->j for i != j and A[i][i] = -(sum of rates out of i),
 * so x' = A x conserves sum(x) (KINETIC -> DERIVATIVE, Section 5.1). */
void orc_kin9_matrix(const double *p, double v, double *A)
{
    static const int edges[12][2] = {
        {0, 1}, {1, 2}, {3, 4}, {4, 5}, {6, 7}, {7, 8},
        {0, 3}, {1, 4}, {2, 5}, {3, 6}, {4, 7}, {5, 8}};
    memset(A, 0, 81 * sizeof(double));
    for (int k = 0; k < 12; ++k) {
        int lo = edges[k][0], hi = edges[k][1];
        double af = p[3 + 4 * k], bf = p[4 + 4 * k];
        double ab = p[5 + 4 * k], bb = p[6 + 4 * k];
        double kf = af * exp(bf * v);  /* lo -> hi */
        double kb = ab * exp(-bb * v); /* hi -> lo */
        A[hi * 9 + lo] += kf;
        A[lo * 9 + lo] -= kf;
        A[lo * 9 + hi] += kb;
        A[hi * 9 + hi] -= kb;
    }
}

/* Dense LU with partial pivoting (the Eigen PartialPivLU method named in
 * Section 5.3), in place on M (row-major n x n) with row permutation perm.
 * Returns the number of row interchanges, or -1 for a zero pivot. */
int orc_lu_pp(int n, double *M, int *perm)
{
    int swaps = 0;
    for (int i = 0; i < n; ++i)
        perm[i] = i;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(M[k * n + k]);
        for (int r = k + 1; r < n; ++r)
            if (fabs(M[r * n + k]) > best) {
                best = fabs(M[r * n + k]);
                piv = r;
            }
        if (best == 0.0)
            return -1;
        if (piv != k) {
            for (int c = 0; c < n; ++c) {
                double t = M[k * n + c];
                M[k * n + c] = M[piv * n + c];
                M[piv * n + c] = t;
            }
            int t = perm[k];
            perm[k] = perm[piv];
            perm[piv] = t;
            ++swaps;
        }
        for (int r = k + 1; r < n; ++r) {
            double l = M[r * n + k] / M[k * n + k];
            M[r * n + k] = l;
            for (int c = k + 1; c < n; ++c)
                M[r * n + c] -= l * M[k * n + c];
        }
    }
    return swaps;
}

/* Solve (P^T L U) x = b using the factors of orc_lu_pp (any n: the
 * intermediate vector is allocated for the call). */
void orc_lu_solve(int n, const double *LU, const int *perm, const double *b,
                  double *x)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        double s = b[perm[i]];
        for (int c = 0; c < i; ++c)
            s -= LU[i * n + c] * y[c];
        y[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int c = i + 1; c < n; ++c)
            s -= LU[i * n + c] * x[c];
        x[i] = s / LU[i * n + i];
    }
    free(y);
}

/* One implicit Euler step of one instance by Newton iteration (Section 5.2
 * derivimplicit, Section 5.3): y0 = x; r = y - x - dt A y; J delta = -r with
 * J = I - dt A; y += delta; stop when max|delta| <= tol or after max_iter
 * updates.  Returns the number of updates; *swaps gets the pivot
 * interchanges of the factorisation. */
int orc_kin9_newton(const double *A, double dt, const double *x, double *y,
                    double tol, int max_iter, int *swaps)
{
    double J[81], r[9], delta[9];
    int perm[9];
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b)
            J[a * 9 + b] = (a == b ? 1.0 : 0.0) - dt * A[a * 9 + b];
    *swaps = orc_lu_pp(9, J, perm);
    for (int a = 0; a < 9; ++a)
        y[a] = x[a];
    int it = 0;
    while (it < max_iter) {
        for (int a = 0; a < 9; ++a) {
            double Ay = 0.0;
            for (int b = 0; b < 9; ++b)
                Ay += A[a * 9 + b] * y[b];
            r[a] = -(y[a] - x[a] - dt * Ay);
        }
        orc_lu_solve(9, J, perm, r, delta);
        double dmax = 0.0;
        for (int a = 0; a < 9; ++a) {
            y[a] += delta[a];
            if (fabs(delta[a]) > dmax)
                dmax = fabs(delta[a]);
        }
        ++it;
        if (dmax <= tol)
            break;
    }
    return it;
}

void orc_kin9_state(int64_t n, const int32_t *ni, const double *v,
                    const double *p, double dt, double *s, double tol,
                    int max_iter, int32_t *iters, int64_t *total_swaps)
{
    int64_t sw_total = 0;
    for (int64_t i = 0; i < n; ++i) {
        double A[81], x[9], y[9];
        int sw = 0;
        orc_kin9_matrix(p, v[ni[i]], A);
        for (int a = 0; a < 9; ++a)
            x[a] = s[a * n + i];
        int it = orc_kin9_newton(A, dt, x, y, tol, max_iter, &sw);
        sw_total += sw;
        if (iters)
            iters[i] = it;
        for (int a = 0; a < 9; ++a)
            s[a * n + i] = y[a];
    }
    if (total_swaps)
        *total_swaps = sw_total;
}

/* Stationary distribution at v: A pi = 0 with sum(pi) = 1, solved as the
 * square system whose last row is replaced by the normalisation. */
int orc_kin9_stationary(const double *p, double v, double *pi)
{
    double A[81], M[81], b[9];
    int perm[9];
    orc_kin9_matrix(p, v, A);
    memcpy(M, A, sizeof(M));
    for (int c = 0; c < 9; ++c)
        M[8 * 9 + c] = 1.0;
    for (int a = 0; a < 9; ++a)
        b[a] = (a == 8) ? 1.0 : 0.0;
    if (orc_lu_pp(9, M, perm) < 0)
        return -1;
    orc_lu_solve(9, M, perm, b, pi);
    return 0;
}

/* ------------------------------------------------ 3-state kinetic scheme */

/* Generator matrix of the 3-state scheme (KINETIC, Section 5.1): edges
 * 0-1, 1-2 and 0-2, each with the forward (lo -> hi) rate af exp(bf v) and
 * the backward rate ab exp(-bb v); params: gbar, e, open, then
 * (af, bf, ab, bb) per edge. */
void orc_kin3_matrix(const double *p, double v, double *A)
{
    static const int edges[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    memset(A, 0, 9 * sizeof(double));
    for (int k = 0; k < 3; ++k) {
        int lo = edges[k][0], hi = edges[k][1];
        double kf = p[3 + 4 * k] * exp(p[4 + 4 * k] * v);
        double kb = p[5 + 4 * k] * exp(-p[6 + 4 * k] * v);
        A[hi * 3 + lo] += kf;
        A[lo * 3 + lo] -= kf;
        A[lo * 3 + hi] += kb;
        A[hi * 3 + hi] -= kb;
    }
}

/* Implicit Euler step of an ns-state linear scheme by the same Newton
 * iteration as the 9-state one (dense LU with partial pivoting of
 * J = I - dt A); for a linear scheme the first update is already the
 * solution and the second is of rounding size. */
int orc_kin_newton_n(int ns, const double *A, double dt, const double *x, double *y,
                     double tol, int max_iter)
{
    double J[64], r[8], delta[8];
    int perm[8];
    if (ns < 1 || ns > 8)
        return -1;
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b)
            J[a * ns + b] = (a == b ? 1.0 : 0.0) - dt * A[a * ns + b];
    orc_lu_pp(ns, J, perm);
    for (int a = 0; a < ns; ++a)
        y[a] = x[a];
    int it = 0;
    while (it < max_iter) {
        for (int a = 0; a < ns; ++a) {
            double Ay = 0.0;
            for (int b = 0; b < ns; ++b)
                Ay += A[a * ns + b] * y[b];
            r[a] = -(y[a] - x[a] - dt * Ay);
        }
        orc_lu_solve(ns, J, perm, r, delta);
        double dmax = 0.0;
        for (int a = 0; a < ns; ++a) {
            y[a] += delta[a];
            if (fabs(delta[a]) > dmax)
                dmax = fabs(delta[a]);
        }
        ++it;
        if (dmax <= tol)
            break;
    }
    return it;
}

/* stationary distribution: last row of A replaced by the normalisation */
int orc_kin_stationary_n(int ns, const double *A, double *pi)
{
    double M[64], b[8];
    int perm[8];
    if (ns < 1 || ns > 8)
        return -1;
    memcpy(M, A, ns * ns * sizeof(double));
    for (int c = 0; c < ns; ++c)
        M[(ns - 1) * ns + c] = 1.0;
    for (int a = 0; a < ns; ++a)
        b[a] = (a == ns - 1) ? 1.0 : 0.0;
    if (orc_lu_pp(ns, M, perm) < 0)
        return -1;
    orc_lu_solve(ns, M, perm, b, pi);
    return 0;
}

/* ------------------------------------------------- calcium accumulation */

/* 2-state calcium accumulation with a buffer (reading of a derivimplicit
 * "cacum"-style mechanism, Section 5.2 / Section 8): y = (cai, cab) [mM],
 *   dcai/dt = -k ica - kf cai (btot - cab) + kb cab - (cai - cai0)/tau
 *   dcab/dt =  kf cai (btot - cab) - kb cab
 * params: k [mM/ms per mA/cm2], tau [ms], cai0 [mM], kf [1/(mM ms)],
 * kb [1/ms], btot [mM].  ica is the node's calcium current of the same step. */
static void cacum_f(const double *p, double ica, const double *y, double *f)
{
    double bind = p[3] * y[0] * (p[5] - y[1]) - p[4] * y[1];
    f[0] = -p[0] * ica - bind - (y[0] - p[2]) / p[1];
    f[1] = bind;
}

static void cacum_jac(const double *p, const double *y, double *Jf)
{
    Jf[0] = -p[3] * (p[5] - y[1]) - 1.0 / p[1];
    Jf[1] = p[3] * y[0] + p[4];
    Jf[2] = p[3] * (p[5] - y[1]);
    Jf[3] = -p[3] * y[0] - p[4];
}

/* One implicit Euler step by Newton's method with the exact Jacobian
 * J = I - dt df/dy and an LU (partial pivot) solve per update. */
int orc_cacum_newton(const double *p, double dt, double ica, const double *x,
                     double *y, double tol, int max_iter)
{
    y[0] = x[0];
    y[1] = x[1];
    int it = 0;
    while (it < max_iter) {
        double f[2], Jf[4], J[4], r[2], delta[2];
        int perm[2];
        cacum_f(p, ica, y, f);
        cacum_jac(p, y, Jf);
        for (int a = 0; a < 2; ++a) {
            r[a] = -(y[a] - x[a] - dt * f[a]);
            for (int b = 0; b < 2; ++b)
                J[a * 2 + b] = (a == b ? 1.0 : 0.0) - dt * Jf[a * 2 + b];
        }
        orc_lu_pp(2, J, perm);
        orc_lu_solve(2, J, perm, r, delta);
        y[0] += delta[0];
        y[1] += delta[1];
        ++it;
        if (fabs(delta[0]) <= tol && fabs(delta[1]) <= tol)
            break;
    }
    return it;
}

/* per-node ion current arrays for the state updates that READ them */
static const double *orc_ion_read[ORC_NION];

void orc_set_ion_read(int ion, const double *arr)
{
    if (ion >= 0 && ion < ORC_NION)
        orc_ion_read[ion] = arr;
}

/* --------------------------------------------------------- per mechanism */

void orc_mech_init(int type, int64_t n, const int32_t *ni, const double *v,
                   const double *p, double *s)
{
    if (type == ORC_TYPE_CACUM) { /* rest: cai0 and the bound buffer at it */
        for (int64_t i = 0; i < n; ++i) {
            s[i] = p[2];
            s[n + i] = p[3] * p[2] * p[5] / (p[3] * p[2] + p[4]);
        }
        return;
    }
    if (type == ORC_TYPE_KIN3) {
        for (int64_t i = 0; i < n; ++i) {
            double A[9], pi[3];
            orc_kin3_matrix(p, v[ni[i]], A);
            orc_kin_stationary_n(3, A, pi);
            for (int a = 0; a < 3; ++a)
                s[a * n + i] = pi[a];
        }
        return;
    }
    if (type == ORC_TYPE_KIN9) {
        for (int64_t i = 0; i < n; ++i) {
            double pi[9];
            orc_kin9_stationary(p, v[ni[i]], pi);
            for (int a = 0; a < 9; ++a)
                s[a * n + i] = pi[a];
        }
    } else {
        cnexp_like_init(type, n, ni, v, p, s);
    }
}

void orc_mech_state(int type, int64_t n, const int32_t *ni, const double *v,
                    const double *p, double dt, double *s, double tol,
                    int max_iter, int32_t *iters)
{
    if (type == ORC_TYPE_KIN9) {
        orc_kin9_state(n, ni, v, p, dt, s, tol, max_iter, iters, NULL);
    } else if (type == ORC_TYPE_KIN3) {
        for (int64_t i = 0; i < n; ++i) {
            double A[9], x[3], y[3];
            orc_kin3_matrix(p, v[ni[i]], A);
            for (int a = 0; a < 3; ++a)
                x[a] = s[a * n + i];
            int it = orc_kin_newton_n(3, A, dt, x, y, tol, max_iter);
            if (iters)
                iters[i] = it;
            for (int a = 0; a < 3; ++a)
                s[a * n + i] = y[a];
        }
    } else if (type == ORC_TYPE_CACUM) {
        const double *ica = orc_ion_read[3];
        for (int64_t i = 0; i < n; ++i) {
            double x[2] = {s[i], s[n + i]}, y[2];
            int it = orc_cacum_newton(p, dt, ica ? ica[ni[i]] : 0.0, x, y, tol, max_iter);
            if (iters)
                iters[i] = it;
            s[i] = y[0];
            s[n + i] = y[1];
        }
    } else {
        cnexp_like_state(type, n, ni, v, p, dt, s);
    }
}

/* ------------------------------------------------------------------ step */

typedef struct {
    int32_t type;
    int32_t ion; /* USEION WRITE tag (0 none, 1 na, 2 k, 3 ca) */
    int64_t n;
    const int32_t *node_index;
    const double *params;
    double *states;
} orc_mech;

/* nsteps time steps of the isolated-compartment network:
 * rhs = d = 0; current update of every mechanism in list order;
 * d += 1e-3 cm/dt (cm in uF/cm2, dt in ms: S/cm2); v += rhs/d unless v is
 * clamped; state update of every mechanism at the new v. */
void orc_step(int n_mechs, const orc_mech *mechs, int64_t n_nodes, double dt,
              double cm, double *v, double *rhs, double *d, int nsteps,
              int clamp_v, double tol, int max_iter)
{
    for (int st = 0; st < nsteps; ++st) {
        for (int64_t k = 0; k < n_nodes; ++k) {
            rhs[k] = 0.0;
            d[k] = 0.0;
        }
        for (int m = 0; m < n_mechs; ++m)
            orc_mech_cur(mechs[m].type, mechs[m].n, mechs[m].node_index, v,
                         mechs[m].params, mechs[m].states, rhs, d);
        for (int64_t k = 0; k < n_nodes; ++k) {
            d[k] += 1e-3 * cm / dt;
            if (!clamp_v)
                v[k] += rhs[k] / d[k];
        }
        for (int m = 0; m < n_mechs; ++m)
            orc_mech_state(mechs[m].type, mechs[m].n, mechs[m].node_index, v,
                           mechs[m].params, dt, mechs[m].states, tol,
                           max_iter, NULL);
    }
}

/* ------------------------------------------------------------- cable */

/* One cable step per cell (reading: NEURON's implicit step with the
 * cable's tree matrix, the "Other" time of Table 2): the membrane system of
 * orc_step plus, for every non-root node i with parent p, the axial
 * conductances ga[i] (per unit area of i) and gb[i] (per unit area of p):
 *   rhs[i] += ga[i] (v[p] - v[i]),  rhs[p] += gb[i] (v[i] - v[p]),
 *   d[i] += ga[i], d[p] += gb[i],   M[i][p] = -ga[i], M[p][i] = -gb[i],
 * then M dv = rhs is solved per cell by the dense partial-pivot LU and
 * v += dv.  Cells are the contiguous node ranges that start at a root
 * (parent -1); parent[i] < i inside a cell. */
void orc_step_cable(int n_mechs, const orc_mech *mechs, int64_t n_nodes,
                    const int32_t *parent, const double *ga, const double *gb,
                    double dt, double cm, double *v, double *rhs, double *d,
                    int nsteps, double tol, int max_iter)
{
    for (int st = 0; st < nsteps; ++st) {
        for (int64_t k = 0; k < n_nodes; ++k) {
            rhs[k] = 0.0;
            d[k] = 0.0;
        }
        for (int m = 0; m < n_mechs; ++m)
            orc_mech_cur(mechs[m].type, mechs[m].n, mechs[m].node_index, v,
                         mechs[m].params, mechs[m].states, rhs, d);
        for (int64_t k = 0; k < n_nodes; ++k)
            d[k] += 1e-3 * cm / dt;
        for (int64_t k = 0; k < n_nodes; ++k) {
            int64_t p = parent[k];
            if (p < 0) continue;
            rhs[k] += ga[k] * (v[p] - v[k]);
            rhs[p] += gb[k] * (v[k] - v[p]);
            d[k] += ga[k];
            d[p] += gb[k];
        }
        int64_t c0 = 0;
        while (c0 < n_nodes) {
            int64_t c1 = c0 + 1;
            while (c1 < n_nodes && parent[c1] >= 0) ++c1;
            int n = (int)(c1 - c0);
            double *M = (double *)calloc((size_t)n * n, sizeof(double));
            double *b = (double *)malloc(sizeof(double) * n);
            double *x = (double *)malloc(sizeof(double) * n);
            int *perm = (int *)malloc(sizeof(int) * n);
            for (int i = 0; i < n; ++i) {
                M[i * n + i] = d[c0 + i];
                b[i] = rhs[c0 + i];
                if (i > 0) {
                    int pp = (int)(parent[c0 + i] - c0);
                    M[i * n + pp] = -ga[c0 + i];
                    M[pp * n + i] = -gb[c0 + i];
                }
            }
            orc_lu_pp(n, M, perm);
            orc_lu_solve(n, M, perm, b, x);
            for (int i = 0; i < n; ++i)
                v[c0 + i] += x[i];
            free(M);
            free(b);
            free(x);
            free(perm);
            c0 = c1;
        }
        for (int m = 0; m < n_mechs; ++m)
            orc_mech_state(mechs[m].type, mechs[m].n, mechs[m].node_index, v,
                           mechs[m].params, dt, mechs[m].states, tol,
                           max_iter, NULL);
    }
}

/* orc_step with ion currents: every step zeroes ion_i[1..3] (where given),
 * accumulates the ion currents of the current update into them, and the
 * state updates that READ an ion (calcium accumulation reads ica) see the
 * same step's values -- the USEION ordering: currents before states. */
void orc_step_ions(int n_mechs, const orc_mech *mechs, int64_t n_nodes, double dt,
                   double cm, double *v, double *rhs, double *d, double *const *ion_i,
                   int nsteps, int clamp_v, double tol, int max_iter)
{
    for (int st = 0; st < nsteps; ++st) {
        for (int64_t k = 0; k < n_nodes; ++k) {
            rhs[k] = 0.0;
            d[k] = 0.0;
            for (int q = 1; q < ORC_NION; ++q)
                if (ion_i[q])
                    ion_i[q][k] = 0.0;
        }
        for (int m = 0; m < n_mechs; ++m) {
            orc_mech_cur(mechs[m].type, mechs[m].n, mechs[m].node_index, v,
                         mechs[m].params, mechs[m].states, rhs, d);
            orc_mech_ion_cur(mechs[m].type, mechs[m].ion, mechs[m].n, mechs[m].node_index,
                             v, mechs[m].params, mechs[m].states, ion_i);
        }
        for (int64_t k = 0; k < n_nodes; ++k) {
            d[k] += 1e-3 * cm / dt;
            if (!clamp_v)
                v[k] += rhs[k] / d[k];
        }
        for (int q = 0; q < ORC_NION; ++q)
            orc_set_ion_read(q, ion_i[q]);
        for (int m = 0; m < n_mechs; ++m)
            orc_mech_state(mechs[m].type, mechs[m].n, mechs[m].node_index, v,
                           mechs[m].params, dt, mechs[m].states, tol, max_iter, NULL);
        for (int q = 0; q < ORC_NION; ++q)
            orc_set_ion_read(q, NULL);
    }
}
