/*
 * ptn_oracle.c -- serial FP64 CPU oracle for the parallel-in-time Newton method
 * for constrained nonlinear MPC (Iacob, Abdulsamad, Saerkkae, arXiv 2409.20027).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code with the CUDA implementation.
 *
 * What it computes (paper sections in brackets):
 *   - the constrained OCP (Sec. II-A, eq. ocp): x_{t+1} = f(x_t,u_t), box constraints
 *     g(x) <= 0, h(u) <= 0, quadratic tracking cost without a 1/2 factor;
 *   - the augmented costs (Sec. III-A): log barrier c^ for IP, penalty c- for ADMM;
 *   - one Newton step (Sec. III, Alg. 4) written as its plain sequential definition:
 *       co-state recursion (eq. co-state-eq, co-state-final),
 *       second-order expansion P, R, M, d (Sec. III-C),
 *       LM-regularised LQR (eq. linearized-ocp-param) solved by the Riccati recursion
 *       (eq. linearized-ocp-bellman) with the feedback law eq. value-fun-feedback,
 *       forward state recursion (eq. closed-loop-dynamics);
 *   - the associative elements and operators of Alg. 1-3 exactly as the paper defines
 *     them (eq. co-states-comb-rule, value-fun-param, value-fun-elem-init,
 *     state-prop-comb-rule), exported so tests can fold them in any association order;
 *   - step acceptance (closed-loop nonlinear rollout, Armijo, Marquardt alpha update),
 *     the primal log-barrier loop (eq. lb-min, lb-step-2) and ADMM
 *     (eq. admm-min ... admm-step-5);
 *   - KKT residuals and the adjoint (envelope theorem + implicit-function VJP).
 *
 * Model derivatives are exact: every discrete step f is evaluated on hyper-dual
 * numbers a + b e1 + c e2 + d e1 e2 (e1^2 = e2^2 = 0), whose e1 part is a directional
 * first derivative and whose e1e2 part is a mixed second derivative.
 *
 * Readings of the paper where it is silent or garbled are marked "reading:".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 32
#define ORC_MAXM 8
#define ORC_MAXW (2 * ORC_MAXN + 2 * ORC_MAXM)
#define ORC_MAXP 8

enum { ORC_PENDULUM = 0, ORC_CARTPOLE = 1, ORC_QUADROTOR = 2, ORC_SYNTH = 3 };
enum { ORC_EULER = 0, ORC_RK4 = 1 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_EINFEAS = -2, ORC_ENOTCONV = -3, ORC_ENUM = -4 };
enum { AUG_NONE = 0, AUG_BARRIER = 1, AUG_ADMM = 2 };

/* Optional user-written terms of the problem statement (Sec. II-A, eq. ocp: a general stage
 * cost l_t, terminal cost l_T and inequality rows g_t(x, u) <= 0), given as callbacks with
 * their derivatives over z = (x, u):
 *   ustage: l_t(x, u); gz (n + m) its gradient and Hz ((n+m) x (n+m), row-major) its
 *           Hessian when the pointers are non-NULL;
 *   uterm:  l_T(x); gx (n), Hx (n x n) likewise;
 *   ucons:  the nc rows g_i(t, x, u) into g (nc); Jz (nc x (n+m)) and Hz (nc x (n+m) x (n+m))
 *           when non-NULL.
 * A user stage / terminal cost replaces the quadratic tracking term; user rows join the
 * box rows in the log barrier (interior point only). */
typedef double (*orc_ustage_fn)(void *ctx, int t, const double *x, const double *u, double *gz, double *Hz);
typedef double (*orc_uterm_fn)(void *ctx, const double *x, double *gx, double *Hx);
typedef void (*orc_ucons_fn)(void *ctx, int t, const double *x, const double *u, double *g, double *Jz,
                             double *Hz);

#define ORC_MAXC 8

typedef struct orc_problem {
    int model, nx, nu, integrator;
    double dt;
    double prm[ORC_MAXP];
    const double *A, *B, *W;         /* synthetic model matrices, row-major */
    const double *Q, *R, *Qf;        /* cost weights, row-major */
    const double *xref, *uref;       /* tracking targets */
    const double *xref_traj;         /* time-varying targets (T+1) x nx, or NULL: xref at every t */
    const double *uref_traj;         /* T x nu, or NULL: uref at every t */
    int T_traj;                      /* horizon of the target trajectories (the terminal index) */
    orc_ustage_fn ustage;            /* user stage cost, or NULL (quadratic tracking) */
    orc_uterm_fn uterm;              /* user terminal cost, or NULL */
    orc_ucons_fn ucons;              /* user inequality rows, or NULL */
    int nc;                          /* number of user rows (<= ORC_MAXC) */
    void *uctx;                      /* passed to the callbacks */
    const double *xlo, *xhi, *ulo, *uhi; /* box bounds; |b| >= 1e300 or non-finite = none */
} orc_problem;

typedef struct orc_options {
    double mu0, zeta, mu_final, tol_inner, tol_final, rho, admm_tol;
    double alpha0, alpha_min, alpha_max, ls_beta, armijo_c1, armijo_eps;
    int max_newton, max_outer, ls_count, admm_fixed_iters;
    int costate_mode; /* 0: co-states by the backward recursion (Sec. III-B);
                         1: multiplier form (dynamics multipliers updated by the LQR duals);
                         2: multiplier form whose multipliers restart from the co-states of
                            the recursion at the start of every Newton sub-problem */
    int update_mode;  /* 0: step accepted on the closed-loop nonlinear rollout (line search);
                         1: the update of Alg. 4 as printed, x <- x + dx, u <- u + du */
} orc_options;

typedef struct orc_aug {
    int kind, nw;
    double mu, rho;
    const double *z, *v; /* ADMM: T x nw row-major */
} orc_aug;

/* ------------------------------------------------------------------ */
/* hyper-dual numbers                                                   */
/* ------------------------------------------------------------------ */
typedef struct { double a, b, c, d; } hd;

static hd hc(double v) { hd r = {v, 0.0, 0.0, 0.0}; return r; }
static hd hadd(hd x, hd y) { hd r = {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; return r; }
static hd hsub(hd x, hd y) { hd r = {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; return r; }
static hd hneg(hd x) { hd r = {-x.a, -x.b, -x.c, -x.d}; return r; }
static hd hscl(hd x, double s) { hd r = {s * x.a, s * x.b, s * x.c, s * x.d}; return r; }
static hd hmul(hd x, hd y)
{
    hd r = {x.a * y.a, x.a * y.b + x.b * y.a, x.a * y.c + x.c * y.a,
            x.a * y.d + x.b * y.c + x.c * y.b + x.d * y.a};
    return r;
}
/* chain rule for a scalar function with value f0, first derivative f1, second f2 */
static hd hfun(hd x, double f0, double f1, double f2)
{
    hd r = {f0, f1 * x.b, f1 * x.c, f1 * x.d + f2 * x.b * x.c};
    return r;
}
static hd hsin(hd x) { return hfun(x, sin(x.a), cos(x.a), -sin(x.a)); }
static hd hcos(hd x) { return hfun(x, cos(x.a), -sin(x.a), -cos(x.a)); }
static hd hrec(hd x) { double i = 1.0 / x.a; return hfun(x, i, -i * i, 2.0 * i * i * i); }
static hd hdiv(hd x, hd y) { return hmul(x, hrec(y)); }
static hd htanh(hd x) { double t = tanh(x.a); return hfun(x, t, 1.0 - t * t, -2.0 * t * (1.0 - t * t)); }

/* ------------------------------------------------------------------ */
/* models: continuous right-hand sides (or the discrete map)            */
/* ------------------------------------------------------------------ */

/* Pendulum (Sec. IV-A): theta'' = -(g/l) sin(theta) - b/(m l^2) theta' + u/(m l^2).
 * prm = [g, l, m, b]; x = (theta, omega). */
static void rhs_pendulum(const hd *p, const hd *x, const hd *u, hd *xd)
{
    hd g = p[0], l = p[1], m = p[2], b = p[3];
    hd ml2 = hmul(m, hmul(l, l));
    xd[0] = x[1];
    xd[1] = hadd(hsub(hneg(hmul(hdiv(g, l), hsin(x[0]))), hmul(hdiv(b, ml2), x[1])), hdiv(u[0], ml2));
}

/* Cart-pole (Sec. IV-B), theta = 0 hanging down.  reading: the paper prints
 * l*theta' inside the cart equation; the dimensionally consistent term
 * (and the one conserving energy) is l*theta'^2.  prm = [m_c, m_p, l, g];
 * x = (p, theta, p', theta'). */
static void rhs_cartpole(const hd *p, const hd *x, const hd *u, hd *xd)
{
    hd mc = p[0], mp = p[1], l = p[2], g = p[3];
    hd s = hsin(x[1]), c = hcos(x[1]), td = x[3];
    hd td2 = hmul(td, td);
    hd den = hadd(mc, hmul(mp, hmul(s, s)));
    hd pdd = hdiv(hadd(u[0], hmul(hmul(mp, s), hadd(hmul(l, td2), hmul(g, c)))), den);
    hd num = hsub(hsub(hneg(hmul(u[0], c)), hmul(hmul(mp, hmul(l, td2)), hmul(c, s))),
                  hmul(hmul(hadd(mc, mp), g), s));
    hd tdd = hdiv(num, hmul(l, den));
    xd[0] = x[2];
    xd[1] = x[3];
    xd[2] = pdd;
    xd[3] = tdd;
}

/* Quadrotor (12 states: position, ZYX Euler angles (roll, pitch, yaw), world
 * velocity, body rates; 4 rotor thrusts).  Newton-Euler rigid body, "+" rotor
 * layout: rotor 1 on +x, 2 on +y, 3 on -x, 4 on -y, yaw torque k_m (f1-f2+f3-f4).
 * prm = [mass, Ixx, Iyy, Izz, arm, k_m, g]. */
static void rhs_quadrotor(const hd *p, const hd *x, const hd *u, hd *xd)
{
    hd mass = p[0], Ixx = p[1], Iyy = p[2], Izz = p[3], arm = p[4], km = p[5], g = p[6];
    hd sph = hsin(x[3]), cph = hcos(x[3]);
    hd sth = hsin(x[4]), cth = hcos(x[4]);
    hd sps = hsin(x[5]), cps = hcos(x[5]);
    hd tth = hdiv(sth, cth);
    hd wx = x[9], wy = x[10], wz = x[11];
    hd fsum = hadd(hadd(u[0], u[1]), hadd(u[2], u[3]));
    /* body z-axis in world frame: third column of Rz(yaw) Ry(pitch) Rx(roll) */
    hd r13 = hadd(hmul(cps, hmul(sth, cph)), hmul(sps, sph));
    hd r23 = hsub(hmul(sps, hmul(sth, cph)), hmul(cps, sph));
    hd r33 = hmul(cth, cph);
    hd am = hdiv(fsum, mass);
    xd[0] = x[6];
    xd[1] = x[7];
    xd[2] = x[8];
    /* Euler-angle rates from body rates */
    xd[3] = hadd(wx, hadd(hmul(hmul(sph, tth), wy), hmul(hmul(cph, tth), wz)));
    xd[4] = hsub(hmul(cph, wy), hmul(sph, wz));
    xd[5] = hdiv(hadd(hmul(sph, wy), hmul(cph, wz)), cth);
    xd[6] = hmul(am, r13);
    xd[7] = hmul(am, r23);
    xd[8] = hsub(hmul(am, r33), g);
    hd tx = hmul(arm, hsub(u[1], u[3]));
    hd ty = hmul(arm, hsub(u[2], u[0]));
    hd tz = hmul(km, hsub(hadd(u[0], u[2]), hadd(u[1], u[3])));
    /* I w' = tau - w x (I w) */
    xd[9] = hdiv(hsub(tx, hmul(hsub(Izz, Iyy), hmul(wy, wz))), Ixx);
    xd[10] = hdiv(hsub(ty, hmul(hsub(Ixx, Izz), hmul(wz, wx))), Iyy);
    xd[11] = hdiv(hsub(tz, hmul(hsub(Iyy, Ixx), hmul(wx, wy))), Izz);
}

static void rhs(const orc_problem *P, const hd *p, const hd *x, const hd *u, hd *xd)
{
    switch (P->model) {
    case ORC_PENDULUM: rhs_pendulum(p, x, u, xd); break;
    case ORC_CARTPOLE: rhs_cartpole(p, x, u, xd); break;
    default: rhs_quadrotor(p, x, u, xd); break;
    }
}

/* One discrete step x+ = f(x,u) on hyper-duals. */
static void step_hd(const orc_problem *P, const hd *p, const hd *x, const hd *u, hd *xn)
{
    int n = P->nx, m = P->nu, i, j;
    if (P->model == ORC_SYNTH) {
        /* x+ = A x + B u + c tanh(W x), c = prm[0] */
        for (i = 0; i < n; i++) {
            hd ax = hc(0.0), wx = hc(0.0);
            for (j = 0; j < n; j++) {
                ax = hadd(ax, hscl(x[j], P->A[i * n + j]));
                wx = hadd(wx, hscl(x[j], P->W[i * n + j]));
            }
            for (j = 0; j < m; j++) ax = hadd(ax, hscl(u[j], P->B[i * m + j]));
            xn[i] = hadd(ax, hmul(p[0], htanh(wx)));
        }
        return;
    }
    double h = P->dt;
    if (P->integrator == ORC_EULER) {
        hd k[ORC_MAXN];
        rhs(P, p, x, u, k);
        for (i = 0; i < n; i++) xn[i] = hadd(x[i], hscl(k[i], h));
        return;
    }
    /* classical RK4 with the control held over the step */
    hd k1[ORC_MAXN], k2[ORC_MAXN], k3[ORC_MAXN], k4[ORC_MAXN], y[ORC_MAXN];
    rhs(P, p, x, u, k1);
    for (i = 0; i < n; i++) y[i] = hadd(x[i], hscl(k1[i], 0.5 * h));
    rhs(P, p, y, u, k2);
    for (i = 0; i < n; i++) y[i] = hadd(x[i], hscl(k2[i], 0.5 * h));
    rhs(P, p, y, u, k3);
    for (i = 0; i < n; i++) y[i] = hadd(x[i], hscl(k3[i], h));
    rhs(P, p, y, u, k4);
    for (i = 0; i < n; i++) {
        hd s = hadd(hadd(k1[i], hscl(k2[i], 2.0)), hadd(hscl(k3[i], 2.0), k4[i]));
        xn[i] = hadd(x[i], hscl(s, h / 6.0));
    }
}

/* Seed helper: z = (x,u) with e1 on component i1 and e2 on component i2 (-1: none);
 * parameter k (-1: none) gets e1 when pk1 != 0 or e2 when pk2 != 0. */
static void eval_seeded(const orc_problem *P, const double *x, const double *u, int i1, int i2,
                        int pk1, int pk2, hd *xn)
{
    int n = P->nx, m = P->nu, i;
    hd hx[ORC_MAXN], hu[ORC_MAXM], hp[ORC_MAXP];
    for (i = 0; i < n; i++) hx[i] = hc(x[i]);
    for (i = 0; i < m; i++) hu[i] = hc(u[i]);
    for (i = 0; i < ORC_MAXP; i++) hp[i] = hc(P->prm[i]);
    if (i1 >= 0) { if (i1 < n) hx[i1].b = 1.0; else hu[i1 - n].b = 1.0; }
    if (i2 >= 0) { if (i2 < n) hx[i2].c = 1.0; else hu[i2 - n].c = 1.0; }
    if (pk1 >= 0) hp[pk1].b = 1.0;
    if (pk2 >= 0) hp[pk2].c = 1.0;
    step_hd(P, hp, hx, hu, xn);
}

/* ---- public model entry points ---- */

void orc_step(const orc_problem *P, const double *x, const double *u, double *xn)
{
    hd r[ORC_MAXN];
    eval_seeded(P, x, u, -1, -1, -1, -1, r);
    for (int i = 0; i < P->nx; i++) xn[i] = r[i].a;
}

/* continuous-time right-hand side (not for the synthetic map); used by the model pins */
void orc_rhs(const orc_problem *P, const double *x, const double *u, double *xd)
{
    hd hx[ORC_MAXN], hu[ORC_MAXM], hp[ORC_MAXP], r[ORC_MAXN];
    for (int i = 0; i < P->nx; i++) hx[i] = hc(x[i]);
    for (int i = 0; i < P->nu; i++) hu[i] = hc(u[i]);
    for (int i = 0; i < ORC_MAXP; i++) hp[i] = hc(P->prm[i]);
    rhs(P, hp, hx, hu, r);
    for (int i = 0; i < P->nx; i++) xd[i] = r[i].a;
}

/* F = df/dx (n x n), G = df/du (n x m), row-major */
void orc_jac(const orc_problem *P, const double *x, const double *u, double *F, double *G)
{
    int n = P->nx, m = P->nu;
    hd r[ORC_MAXN];
    for (int j = 0; j < n + m; j++) {
        eval_seeded(P, x, u, j, -1, -1, -1, r);
        for (int i = 0; i < n; i++) {
            if (j < n) F[i * n + j] = r[i].b;
            else G[i * m + (j - n)] = r[i].b;
        }
    }
}

/* Second-order contraction of Sec. III-C: (lam . f_zz)_{ij} = sum_k lam_k d2 f_k / dz_i dz_j,
 * split into Hxx (n x n), Hxu (n x m), Huu (m x m). */
void orc_hess(const orc_problem *P, const double *x, const double *u, const double *lam,
              double *Hxx, double *Hxu, double *Huu)
{
    int n = P->nx, m = P->nu, K = n + m;
    hd r[ORC_MAXN];
    for (int i = 0; i < K; i++)
        for (int j = i; j < K; j++) {
            eval_seeded(P, x, u, i, j, -1, -1, r);
            double h = 0.0;
            for (int k = 0; k < n; k++) h += lam[k] * r[k].d;
            if (i < n && j < n) { Hxx[i * n + j] = h; Hxx[j * n + i] = h; }
            else if (i < n) Hxu[i * m + (j - n)] = h;
            else { Huu[(i - n) * m + (j - n)] = h; Huu[(j - n) * m + (i - n)] = h; }
        }
}

/* df/dprm (n x ORC_MAXP) */
void orc_param_jac(const orc_problem *P, const double *x, const double *u, double *dfdp)
{
    hd r[ORC_MAXN];
    for (int k = 0; k < ORC_MAXP; k++) {
        eval_seeded(P, x, u, -1, -1, k, -1, r);
        for (int i = 0; i < P->nx; i++) dfdp[i * ORC_MAXP + k] = r[i].b;
    }
}

/* d2 (lam^T f) / dz dprm_k : Hzp is (n+m) x ORC_MAXP */
void orc_param_hess(const orc_problem *P, const double *x, const double *u, const double *lam,
                    double *Hzp)
{
    int n = P->nx, m = P->nu;
    hd r[ORC_MAXN];
    for (int j = 0; j < n + m; j++)
        for (int k = 0; k < ORC_MAXP; k++) {
            eval_seeded(P, x, u, j, -1, -1, k, r);
            double h = 0.0;
            for (int i = 0; i < n; i++) h += lam[i] * r[i].d;
            Hzp[j * ORC_MAXP + k] = h;
        }
}

/* ------------------------------------------------------------------ */
/* small dense linear algebra (row-major)                              */
/* ------------------------------------------------------------------ */

/* C = A (r x k) * B (k x c) */
static void mm(int r, int k, int c, const double *A, const double *B, double *C)
{
    for (int i = 0; i < r; i++)
        for (int j = 0; j < c; j++) {
            double s = 0.0;
            for (int l = 0; l < k; l++) s += A[i * k + l] * B[l * c + j];
            C[i * c + j] = s;
        }
}
/* C = A^T B, A is k x r, B is k x c */
static void mtm(int r, int k, int c, const double *A, const double *B, double *C)
{
    for (int i = 0; i < r; i++)
        for (int j = 0; j < c; j++) {
            double s = 0.0;
            for (int l = 0; l < k; l++) s += A[l * r + i] * B[l * c + j];
            C[i * c + j] = s;
        }
}
static void transpose(int r, int c, const double *A, double *At)
{
    for (int i = 0; i < r; i++)
        for (int j = 0; j < c; j++) At[j * r + i] = A[i * c + j];
}

/* Cholesky A = L L^T; returns 0 on success, 1 if A is not positive definite */
static int chol(int n, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int k = 0; k < j; k++) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0) || !isfinite(s)) return 1;
        double d = sqrt(s);
        L[j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int k = 0; k < j; k++) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / d;
        }
    }
    return 0;
}
/* solve (L L^T) X = B in place, B is n x c */
static void chol_solve(int n, int c, const double *L, double *B)
{
    for (int col = 0; col < c; col++) {
        for (int i = 0; i < n; i++) {
            double s = B[i * c + col];
            for (int k = 0; k < i; k++) s -= L[i * n + k] * B[k * c + col];
            B[i * c + col] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = B[i * c + col];
            for (int k = i + 1; k < n; k++) s -= L[k * n + i] * B[k * c + col];
            B[i * c + col] = s / L[i * n + i];
        }
    }
}
/* LU with partial pivoting; solve A X = B in place (B n x c). Returns 1 if singular. */
static int lu_solve(int n, int c, const double *A_in, double *B)
{
    double A[ORC_MAXN * ORC_MAXN];
    memcpy(A, A_in, sizeof(double) * n * n);
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int i = k + 1; i < n; i++)
            if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
        if (!(fabs(A[p * n + k]) > 0.0) || !isfinite(A[p * n + k])) return 1;
        if (p != k) {
            for (int j = 0; j < n; j++) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
            for (int j = 0; j < c; j++) { double t = B[k * c + j]; B[k * c + j] = B[p * c + j]; B[p * c + j] = t; }
        }
        for (int i = k + 1; i < n; i++) {
            double f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; j++) A[i * n + j] -= f * A[k * n + j];
            for (int j = 0; j < c; j++) B[i * c + j] -= f * B[k * c + j];
        }
    }
    for (int j = 0; j < c; j++)
        for (int i = n - 1; i >= 0; i--) {
            double s = B[i * c + j];
            for (int k = i + 1; k < n; k++) s -= A[i * n + k] * B[k * c + j];
            B[i * c + j] = s / A[i * n + i];
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* constraints, stage and terminal costs                                */
/* ------------------------------------------------------------------ */

/* Constraint rows w_r = sgn_r * (z_k - bnd_r) <= 0; state rows first (per component:
 * upper then lower), then control rows.  reading: the paper sizes g and h as d_x and
 * d_u rows; any number of box rows is allowed here. */
typedef struct {
    int nw;
    int isx[ORC_MAXW], idx[ORC_MAXW];
    double sgn[ORC_MAXW], bnd[ORC_MAXW];
} rows_t;

static int has_bound(const double *b, int i) { return b && isfinite(b[i]) && fabs(b[i]) < 1e300; }

static void build_rows(const orc_problem *P, rows_t *R)
{
    int k = 0;
    for (int i = 0; i < P->nx; i++) {
        if (has_bound(P->xhi, i)) { R->isx[k] = 1; R->idx[k] = i; R->sgn[k] = 1.0; R->bnd[k] = P->xhi[i]; k++; }
        if (has_bound(P->xlo, i)) { R->isx[k] = 1; R->idx[k] = i; R->sgn[k] = -1.0; R->bnd[k] = P->xlo[i]; k++; }
    }
    for (int i = 0; i < P->nu; i++) {
        if (has_bound(P->uhi, i)) { R->isx[k] = 0; R->idx[k] = i; R->sgn[k] = 1.0; R->bnd[k] = P->uhi[i]; k++; }
        if (has_bound(P->ulo, i)) { R->isx[k] = 0; R->idx[k] = i; R->sgn[k] = -1.0; R->bnd[k] = P->ulo[i]; k++; }
    }
    R->nw = k;
}

int orc_num_rows(const orc_problem *P)
{
    rows_t R;
    build_rows(P, &R);
    return R.nw;
}

static double row_value(const rows_t *R, int r, const double *x, const double *u)
{
    double zk = R->isx[r] ? x[R->idx[r]] : u[R->idx[r]];
    return R->sgn[r] * (zk - R->bnd[r]);
}

void orc_constraints(const orc_problem *P, const double *x, const double *u, double *w)
{
    rows_t R;
    build_rows(P, &R);
    for (int r = 0; r < R.nw; r++) w[r] = row_value(&R, r, x, u);
}

/* tracking targets at step t (the stage cost l_t of Sec. II-A may vary with t) */
static const double *xref_at(const orc_problem *P, int t)
{
    return P->xref_traj ? P->xref_traj + (size_t)t * P->nx : P->xref;
}
static const double *uref_at(const orc_problem *P, int t)
{
    return P->uref_traj ? P->uref_traj + (size_t)t * P->nu : P->uref;
}

/* Stage cost l_t + c_t at step t (Sec. III-A).  *infeas is set when a barrier row is
 * not strictly negative. */
static double stage_cost(const orc_problem *P, const rows_t *R, const orc_aug *G, int t,
                         const double *x, const double *u, int *infeas, double *lonly)
{
    int n = P->nx, m = P->nu;
    double ex[ORC_MAXN], eu[ORC_MAXM], l = 0.0;
    if (P->ustage) {
        l = P->ustage(P->uctx, t, x, u, NULL, NULL);
    } else {
        const double *xr = xref_at(P, t), *ur = uref_at(P, t);
        for (int i = 0; i < n; i++) ex[i] = x[i] - xr[i];
        for (int i = 0; i < m; i++) eu[i] = u[i] - ur[i];
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) l += ex[i] * P->Q[i * n + j] * ex[j];
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) l += eu[i] * P->R[i * m + j] * eu[j];
    }
    if (lonly) *lonly = l;
    if (P->ucons && P->nc > 0 && G->kind == AUG_BARRIER) {  /* user rows: the IP method */
        double g[ORC_MAXC];
        P->ucons(P->uctx, t, x, u, g, NULL, NULL);
        for (int i = 0; i < P->nc; i++) {
            if (!(g[i] < 0.0)) { *infeas = 1; return INFINITY; }
            l -= G->mu * log(-g[i]);
        }
    }
    double c = 0.0;
    for (int r = 0; r < R->nw; r++) {
        double w = row_value(R, r, x, u);
        if (G->kind == AUG_BARRIER) {
            if (!(w < 0.0)) { *infeas = 1; return INFINITY; }
            c -= G->mu * log(-w);
        } else if (G->kind == AUG_ADMM) {
            double q = w - G->z[t * R->nw + r] + G->v[t * R->nw + r] / G->rho;
            c += 0.5 * G->rho * q * q;
        }
    }
    return l + c;
}

/* Gradients and Hessians of l_t + c_t with respect to x and u. */
static void stage_derivs(const orc_problem *P, const rows_t *R, const orc_aug *G, int t,
                         const double *x, const double *u, double *lx, double *lu, double *lxx,
                         double *lxu, double *luu)
{
    int n = P->nx, m = P->nu, K = n + m;
    if (P->ustage) {
        double gz[ORC_MAXN + ORC_MAXM], Hz[(ORC_MAXN + ORC_MAXM) * (ORC_MAXN + ORC_MAXM)];
        P->ustage(P->uctx, t, x, u, gz, Hz);
        for (int i = 0; i < n; i++) {
            lx[i] = gz[i];
            for (int j = 0; j < n; j++) lxx[i * n + j] = Hz[i * K + j];
            for (int j = 0; j < m; j++) lxu[i * m + j] = Hz[i * K + n + j];
        }
        for (int i = 0; i < m; i++) {
            lu[i] = gz[n + i];
            for (int j = 0; j < m; j++) luu[i * m + j] = Hz[(n + i) * K + n + j];
        }
    } else {
        const double *xr = xref_at(P, t), *ur = uref_at(P, t);
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int j = 0; j < n; j++) s += (P->Q[i * n + j] + P->Q[j * n + i]) * (x[j] - xr[j]);
            lx[i] = s;
            for (int j = 0; j < n; j++) lxx[i * n + j] = P->Q[i * n + j] + P->Q[j * n + i];
            for (int j = 0; j < m; j++) lxu[i * m + j] = 0.0;
        }
        for (int i = 0; i < m; i++) {
            double s = 0.0;
            for (int j = 0; j < m; j++) s += (P->R[i * m + j] + P->R[j * m + i]) * (u[j] - ur[j]);
            lu[i] = s;
            for (int j = 0; j < m; j++) luu[i * m + j] = P->R[i * m + j] + P->R[j * m + i];
        }
    }
    if (P->ucons && P->nc > 0 && G->kind == AUG_BARRIER) {
        /* -mu log(-g): gradient mu grad(g) / (-g), Hessian mu (grad g grad g^T / g^2 + Hess(g) / (-g)) */
        double g[ORC_MAXC], Jz[ORC_MAXC * (ORC_MAXN + ORC_MAXM)],
            Hz[ORC_MAXC * (ORC_MAXN + ORC_MAXM) * (ORC_MAXN + ORC_MAXM)];
        P->ucons(P->uctx, t, x, u, g, Jz, Hz);
        for (int c = 0; c < P->nc; c++) {
            const double a = G->mu / (-g[c]), b = G->mu / (g[c] * g[c]);
            const double *J = Jz + c * K, *H = Hz + (size_t)c * K * K;
            for (int i = 0; i < K; i++) {
                if (i < n) lx[i] += a * J[i]; else lu[i - n] += a * J[i];
                for (int j = 0; j < K; j++) {
                    const double h = b * J[i] * J[j] + a * H[i * K + j];
                    if (i < n && j < n) lxx[i * n + j] += h;
                    else if (i < n) lxu[i * m + (j - n)] += h;
                    else if (j >= n) luu[(i - n) * m + (j - n)] += h;
                }
            }
        }
    }
    for (int r = 0; r < R->nw; r++) {
        double w = row_value(R, r, x, u), sg = R->sgn[r], g1, g2;
        if (G->kind == AUG_BARRIER) {
            /* d/dz [-mu log(-w)] = mu sg / (-w);  d2 = mu sg^2 / w^2 */
            g1 = G->mu * sg / (-w);
            g2 = G->mu * sg * sg / (w * w);
        } else if (G->kind == AUG_ADMM) {
            double q = w - G->z[t * R->nw + r] + G->v[t * R->nw + r] / G->rho;
            g1 = G->rho * q * sg;
            g2 = G->rho * sg * sg;
        } else continue;
        int k = R->idx[r];
        if (R->isx[r]) { lx[k] += g1; lxx[k * n + k] += g2; }
        else { lu[k] += g1; luu[k * m + k] += g2; }
    }
}

static double terminal_cost(const orc_problem *P, const double *x)
{
    int n = P->nx;
    if (P->uterm) return P->uterm(P->uctx, x, NULL, NULL);
    const double *xr = xref_at(P, P->T_traj);
    double l = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) l += (x[i] - xr[i]) * P->Qf[i * n + j] * (x[j] - xr[j]);
    return l;
}
static void terminal_grad(const orc_problem *P, const double *x, double *g, double *H)
{
    int n = P->nx;
    if (P->uterm) {
        double Hx[ORC_MAXN * ORC_MAXN];
        P->uterm(P->uctx, x, g, Hx);
        if (H) memcpy(H, Hx, sizeof(double) * n * n);
        return;
    }
    const double *xr = xref_at(P, P->T_traj);
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int j = 0; j < n; j++) s += (P->Qf[i * n + j] + P->Qf[j * n + i]) * (x[j] - xr[j]);
        g[i] = s;
        if (H) for (int j = 0; j < n; j++) H[i * n + j] = P->Qf[i * n + j] + P->Qf[j * n + i];
    }
}

/* J_c of Sec. III-A over a trajectory; returns INFINITY when infeasible for the barrier.
 * Also returns the un-augmented cost J in *Jplain when non-NULL. */
static double traj_cost(const orc_problem *P, const rows_t *R, const orc_aug *G, int T,
                        const double *x, const double *u, double *Jplain)
{
    int n = P->nx, m = P->nu, inf = 0;
    double J = 0.0, Jl = 0.0, l;
    for (int t = 0; t < T; t++) {
        J += stage_cost(P, R, G, t, x + t * n, u + t * m, &inf, &l);
        Jl += l;
        if (inf) return INFINITY;
    }
    double lt = terminal_cost(P, x + T * n);
    if (Jplain) *Jplain = Jl + lt;
    return J + lt;
}

double orc_cost(const orc_problem *P, const orc_aug *G, int T, const double *x, const double *u,
                double *Jplain)
{
    rows_t R;
    build_rows(P, &R);
    return traj_cost(P, &R, G, T, x, u, Jplain);
}

/* open-loop rollout x_{t+1} = f(x_t, u_t), x_1 = x0 (eq. ocp) */
void orc_rollout(const orc_problem *P, const double *x0, const double *u, int T, double *x)
{
    int n = P->nx, m = P->nu;
    memcpy(x, x0, sizeof(double) * n);
    for (int t = 0; t < T; t++) orc_step(P, x + t * n, u + t * m, x + (t + 1) * n);
}

/* ------------------------------------------------------------------ */
/* one Newton step, sequential definition (Sec. III)                    */
/* ------------------------------------------------------------------ */

typedef struct {
    double *F, *G;          /* T x n*n, T x n*m : Jacobians at the nominal */
    double *lam, *d;        /* (T+1) x n, T x m */
    double *Pm, *Mm, *Rm;   /* T+1 x n*n (last = P_{N+1}), T x n*m, T x m*m */
    double *S, *s;          /* (T+1) x n*n, (T+1) x n */
    double *Gam, *gam;      /* T x m*n, T x m */
    double *dx, *du;        /* (T+1) x n, T x m */
    double G1, G2;
} newton_ws;

static void ws_alloc(newton_ws *W, int T, int n, int m)
{
    W->F = calloc((size_t)T * n * n + 1, sizeof(double));
    W->G = calloc((size_t)T * n * m + 1, sizeof(double));
    W->lam = calloc((size_t)(T + 1) * n, sizeof(double));
    W->d = calloc((size_t)T * m + 1, sizeof(double));
    W->Pm = calloc((size_t)(T + 1) * n * n, sizeof(double));
    W->Mm = calloc((size_t)T * n * m + 1, sizeof(double));
    W->Rm = calloc((size_t)T * m * m + 1, sizeof(double));
    W->S = calloc((size_t)(T + 1) * n * n, sizeof(double));
    W->s = calloc((size_t)(T + 1) * n, sizeof(double));
    W->Gam = calloc((size_t)T * m * n + 1, sizeof(double));
    W->gam = calloc((size_t)T * m + 1, sizeof(double));
    W->dx = calloc((size_t)(T + 1) * n, sizeof(double));
    W->du = calloc((size_t)T * m + 1, sizeof(double));
}
static void ws_free(newton_ws *W)
{
    free(W->F); free(W->G); free(W->lam); free(W->d); free(W->Pm); free(W->Mm); free(W->Rm);
    free(W->S); free(W->s); free(W->Gam); free(W->gam); free(W->dx); free(W->du);
}

/* Co-state pass (eq. co-state-eq and co-state-final):
 *   lam_{N+1} = dl_{N+1}/dx,  lam_t = dl_t/dx + dc_t/dx + F_t^T lam_{t+1},
 * and the control gradient d_t = dH_t/du (Sec. III-C). Returns max_t |d_t|_inf. */
static double costate_pass(const orc_problem *P, const rows_t *R, const orc_aug *G, int T,
                           const double *x, const double *u, newton_ws *W)
{
    int n = P->nx, m = P->nu;
    double lx[ORC_MAXN], lu[ORC_MAXM], lxx[ORC_MAXN * ORC_MAXN], lxu[ORC_MAXN * ORC_MAXM],
        luu[ORC_MAXM * ORC_MAXM];
    terminal_grad(P, x + T * n, W->lam + T * n, NULL);
    double dmax = 0.0;
    for (int t = T - 1; t >= 0; t--) {
        double *F = W->F + (size_t)t * n * n, *Gm = W->G + (size_t)t * n * m;
        orc_jac(P, x + t * n, u + t * m, F, Gm);
        stage_derivs(P, R, G, t, x + t * n, u + t * m, lx, lu, lxx, lxu, luu);
        const double *ln = W->lam + (t + 1) * n;
        for (int i = 0; i < n; i++) {
            double s = lx[i];
            for (int k = 0; k < n; k++) s += F[k * n + i] * ln[k];
            W->lam[t * n + i] = s;
        }
        for (int i = 0; i < m; i++) {
            double s = lu[i];
            for (int k = 0; k < n; k++) s += Gm[k * m + i] * ln[k];
            W->d[t * m + i] = s;
            if (!(fabs(s) <= dmax)) dmax = isfinite(s) ? fabs(s) : INFINITY;
        }
    }
    return dmax;
}

/* Multiplier form of the first-order terms (a variant of the method, not in the paper:
 * it replaces the co-state recursion of Sec. III-B, whose products of F_t^T grow without
 * bound on long horizons of an unstable system).  nu holds multipliers of the dynamics
 * constraints; with the Lagrangian
 *   L = sum_t l_t(x_t, u_t) + l_{N+1}(x_{N+1}) + sum_t nu_{t+1}^T (f(x_t, u_t) - x_{t+1})
 * the gradients are d_t = dL/du_t = dl_t/du + G_t^T nu_{t+1} and
 *   q_t = dL/dx_t = dl_t/dx + F_t^T nu_{t+1} - nu_t   (t = 2..N),
 *   q_{N+1} = dl_{N+1}/dx - nu_{N+1},   q_1 = 0 (x_1 is fixed).
 * Each term is local in t: no recursion.  W->lam is set to nu, so the second-order terms
 * contract the model Hessians with nu_{t+1}.  At q = 0, nu is the co-state of Sec. III-B.
 * Returns max(max_t |d_t|_inf, max_t |q_t|_inf). */
static double multiplier_pass(const orc_problem *P, const rows_t *R, const orc_aug *G, int T,
                              const double *x, const double *u, double *nu, newton_ws *W,
                              double *q)
{
    int n = P->nx, m = P->nu;
    double lx[ORC_MAXN], lu[ORC_MAXM], lxx[ORC_MAXN * ORC_MAXN], lxu[ORC_MAXN * ORC_MAXM],
        luu[ORC_MAXM * ORC_MAXM], gT[ORC_MAXN];
    memcpy(W->lam, nu, sizeof(double) * (T + 1) * n);
    double r = 0.0;
    terminal_grad(P, x + T * n, gT, NULL);
    for (int i = 0; i < n; i++) {
        q[T * n + i] = gT[i] - nu[T * n + i];
        if (!(fabs(q[T * n + i]) <= r)) r = isfinite(q[T * n + i]) ? fabs(q[T * n + i]) : INFINITY;
    }
    for (int t = 0; t < T; t++) {
        double *F = W->F + (size_t)t * n * n, *Gm = W->G + (size_t)t * n * m;
        orc_jac(P, x + t * n, u + t * m, F, Gm);
        stage_derivs(P, R, G, t, x + t * n, u + t * m, lx, lu, lxx, lxu, luu);
        const double *nn = nu + (t + 1) * n;
        for (int i = 0; i < n; i++) {
            double v = lx[i];
            for (int k = 0; k < n; k++) v += F[k * n + i] * nn[k];
            if (t == 0) {
                /* x_1 is fixed: its multiplier is defined by one step of the co-state
                 * relation (it is the gradient of the cost in x0), q_1 = 0 */
                nu[i] = v;
                W->lam[i] = v;
                q[i] = 0.0;
                continue;
            }
            v -= nu[t * n + i];
            q[t * n + i] = v;
            if (!(fabs(v) <= r)) r = isfinite(v) ? fabs(v) : INFINITY;
        }
        for (int i = 0; i < m; i++) {
            double v = lu[i];
            for (int k = 0; k < n; k++) v += Gm[k * m + i] * nn[k];
            W->d[t * m + i] = v;
            if (!(fabs(v) <= r)) r = isfinite(v) ? fabs(v) : INFINITY;
        }
    }
    return r;
}

/* Second-order expansion of the Lagrangian (Sec. III-C):
 *   P_t = l_xx + c_xx + lam_{t+1}.f_xx,  M_t = l_xu + c_xu + lam_{t+1}.f_xu,
 *   R_t = l_uu + c_uu + lam_{t+1}.f_uu,  P_{N+1} = d2 l_{N+1}/dx2.  */
static void quadratize(const orc_problem *P, const rows_t *R, const orc_aug *G, int T,
                       const double *x, const double *u, newton_ws *W)
{
    int n = P->nx, m = P->nu;
    double lx[ORC_MAXN], lu[ORC_MAXM], lxx[ORC_MAXN * ORC_MAXN], lxu[ORC_MAXN * ORC_MAXM],
        luu[ORC_MAXM * ORC_MAXM], hxx[ORC_MAXN * ORC_MAXN], hxu[ORC_MAXN * ORC_MAXM],
        huu[ORC_MAXM * ORC_MAXM];
    for (int t = 0; t < T; t++) {
        stage_derivs(P, R, G, t, x + t * n, u + t * m, lx, lu, lxx, lxu, luu);
        orc_hess(P, x + t * n, u + t * m, W->lam + (t + 1) * n, hxx, hxu, huu);
        for (int i = 0; i < n * n; i++) W->Pm[(size_t)t * n * n + i] = lxx[i] + hxx[i];
        for (int i = 0; i < n * m; i++) W->Mm[(size_t)t * n * m + i] = lxu[i] + hxu[i];
        for (int i = 0; i < m * m; i++) W->Rm[(size_t)t * m * m + i] = luu[i] + huu[i];
    }
    double g[ORC_MAXN];
    terminal_grad(P, x + T * n, g, W->Pm + (size_t)T * n * n);
}

/* Riccati recursion for the regularised LQR of eq. linearized-ocp / linearized-ocp-param
 * with R~ = R + alpha I, giving S_t, s_t (V_t = 1/2 dx^T S dx + dx^T s) and the feedback of
 * eq. value-fun-feedback (reading: Q^{-1} M_t^T, the printed Q^{-1} M_t does not conform).
 * qx (T+1 x n, may be NULL) adds a linear state term q_t^T dx_t to psi_t (used by the
 * adjoint; the Newton step has none).  Returns 1 if some R~_t or Q_t is not positive
 * definite: the parallel element init needs R~_t^{-1} and the feedback needs Q_t^{-1}. */
static int riccati(int n, int m, int T, newton_ws *W, double alpha, const double *qx)
{
    double Rt[ORC_MAXM * ORC_MAXM], L[ORC_MAXM * ORC_MAXM], SG[ORC_MAXN * ORC_MAXM],
        SF[ORC_MAXN * ORC_MAXN], Quu[ORC_MAXM * ORC_MAXM], Qux[ORC_MAXM * ORC_MAXN],
        Qu[ORC_MAXM], Qxx[ORC_MAXN * ORC_MAXN], Qx[ORC_MAXN], rhs[ORC_MAXM * (ORC_MAXN + 1)];
    memcpy(W->S + (size_t)T * n * n, W->Pm + (size_t)T * n * n, sizeof(double) * n * n);
    for (int i = 0; i < n; i++) W->s[T * n + i] = qx ? qx[T * n + i] : 0.0;
    for (int t = T - 1; t >= 0; t--) {
        const double *F = W->F + (size_t)t * n * n, *Gm = W->G + (size_t)t * n * m;
        const double *Sn = W->S + (size_t)(t + 1) * n * n, *sn = W->s + (t + 1) * n;
        for (int i = 0; i < m * m; i++) Rt[i] = W->Rm[(size_t)t * m * m + i];
        for (int i = 0; i < m; i++) Rt[i * m + i] += alpha;
        if (chol(m, Rt, L)) return 1;
        mm(n, n, m, Sn, Gm, SG);       /* S G */
        mm(n, n, n, Sn, F, SF);        /* S F */
        mtm(m, n, m, Gm, SG, Quu);     /* G^T S G */
        for (int i = 0; i < m * m; i++) Quu[i] += Rt[i];
        mtm(m, n, n, Gm, SF, Qux);     /* G^T S F */
        for (int i = 0; i < m; i++)
            for (int j = 0; j < n; j++) Qux[i * n + j] += W->Mm[(size_t)t * n * m + j * m + i];
        for (int i = 0; i < m; i++) {
            double s = W->d[t * m + i];
            for (int k = 0; k < n; k++) s += Gm[k * m + i] * sn[k];
            Qu[i] = s;
        }
        mtm(n, n, n, F, SF, Qxx);      /* F^T S F */
        for (int i = 0; i < n * n; i++) Qxx[i] += W->Pm[(size_t)t * n * n + i];
        for (int i = 0; i < n; i++) {
            double s = qx ? qx[t * n + i] : 0.0;
            for (int k = 0; k < n; k++) s += F[k * n + i] * sn[k];
            Qx[i] = s;
        }
        if (chol(m, Quu, L)) return 1;
        /* [Gam | gam] = -Quu^{-1} [Qux | Qu] */
        for (int i = 0; i < m; i++) {
            for (int j = 0; j < n; j++) rhs[i * (n + 1) + j] = Qux[i * n + j];
            rhs[i * (n + 1) + n] = Qu[i];
        }
        chol_solve(m, n + 1, L, rhs);
        double *Gam = W->Gam + (size_t)t * m * n, *gam = W->gam + t * m;
        for (int i = 0; i < m; i++) {
            for (int j = 0; j < n; j++) Gam[i * n + j] = -rhs[i * (n + 1) + j];
            gam[i] = -rhs[i * (n + 1) + n];
        }
        /* S_t = Qxx + Qux^T Gam, s_t = Qx + Qux^T gam */
        double *S = W->S + (size_t)t * n * n, *s = W->s + t * n;
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < n; j++) {
                double v = Qxx[i * n + j];
                for (int k = 0; k < m; k++) v += Qux[k * n + i] * Gam[k * n + j];
                S[i * n + j] = v;
            }
            double v = Qx[i];
            for (int k = 0; k < m; k++) v += Qux[k * n + i] * gam[k];
            s[i] = v;
        }
    }
    return 0;
}

/* Forward pass (eq. closed-loop-dynamics): dx_1 = 0, du_t = Gam_t dx_t + gam_t,
 * dx_{t+1} = F_t dx_t + G_t du_t; also the model terms
 *   G1 = sum_t d_t^T du_t,
 *   G2 = 1/2 [ sum_t (dx^T P dx + 2 dx^T M du + du^T R du) + dx_{N+1}^T P_{N+1} dx_{N+1} ]. */
static void forward_pass(int n, int m, int T, newton_ws *W)
{
    memset(W->dx, 0, sizeof(double) * n);
    double G1 = 0.0, G2 = 0.0;
    for (int t = 0; t < T; t++) {
        const double *F = W->F + (size_t)t * n * n, *Gm = W->G + (size_t)t * n * m;
        const double *Gam = W->Gam + (size_t)t * m * n, *gam = W->gam + t * m;
        const double *dx = W->dx + t * n;
        double *du = W->du + t * m, *dxn = W->dx + (t + 1) * n;
        for (int i = 0; i < m; i++) {
            double v = gam[i];
            for (int j = 0; j < n; j++) v += Gam[i * n + j] * dx[j];
            du[i] = v;
        }
        for (int i = 0; i < n; i++) {
            double v = 0.0;
            for (int j = 0; j < n; j++) v += F[i * n + j] * dx[j];
            for (int j = 0; j < m; j++) v += Gm[i * m + j] * du[j];
            dxn[i] = v;
        }
        const double *Pt = W->Pm + (size_t)t * n * n, *Mt = W->Mm + (size_t)t * n * m,
                     *Rt = W->Rm + (size_t)t * m * m;
        for (int i = 0; i < m; i++) G1 += W->d[t * m + i] * du[i];
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) G2 += 0.5 * dx[i] * Pt[i * n + j] * dx[j];
        for (int i = 0; i < n; i++)
            for (int j = 0; j < m; j++) G2 += dx[i] * Mt[i * m + j] * du[j];
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) G2 += 0.5 * du[i] * Rt[i * m + j] * du[j];
    }
    const double *PT = W->Pm + (size_t)T * n * n, *dxT = W->dx + T * n;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) G2 += 0.5 * dxT[i] * PT[i * n + j] * dxT[j];
    W->G1 = G1;
    W->G2 = G2;
}

/* Multiplier form, first-order model term: G1 += sum_t q_t^T dx_t.  The multiplier
 * terms of the Lagrangian telescope away along the linearised dynamics (dx_1 = 0), so
 * G1 stays the cost's directional derivative along (dx, du). */
static void mult_g1(int n, int T, const double *q, newton_ws *W)
{
    for (int t = 1; t <= T; t++)
        for (int i = 0; i < n; i++) W->G1 += q[t * n + i] * W->dx[t * n + i];
}

/* Multiplier form, dual step: dnu_t = S_t dx_t + s_t, the gradient of the LQR value
 * function at dx_t (the multiplier of the linearised dynamics into step t). */
static void mult_dual(int n, int T, const newton_ws *W, double *dnu)
{
    for (int t = 0; t <= T; t++) {
        const double *S = W->S + (size_t)t * n * n, *sv = W->s + t * n, *dx = W->dx + t * n;
        for (int i = 0; i < n; i++) {
            double v = sv[i];
            for (int j = 0; j < n; j++) v += S[i * n + j] * dx[j];
            dnu[t * n + i] = v;
        }
    }
}

/* Public: one full Newton direction at the nominal (x, u) for regularisation alpha.
 * Outputs (any may be NULL): lam (T+1)xn, d Txm, S (T+1)xnxn, s (T+1)xn, Gam Txmxn,
 * gam Txm, dx (T+1)xn, du Txm, P (T+1)xnxn, M Txnxm, R Txmxm, F Txnxn, G Txnxm, g12[2].
 * Returns 0, or 1 when R~ or Q is not positive definite. */
int orc_newton_direction(const orc_problem *P, const orc_aug *G, int T, const double *x,
                         const double *u, double alpha, double *lam, double *d, double *S,
                         double *s, double *Gam, double *gam, double *dx, double *du, double *Pm,
                         double *Mm, double *Rm, double *F, double *Gm, double *g12)
{
    int n = P->nx, m = P->nu;
    rows_t R;
    build_rows(P, &R);
    newton_ws W;
    ws_alloc(&W, T, n, m);
    costate_pass(P, &R, G, T, x, u, &W);
    quadratize(P, &R, G, T, x, u, &W);
    int st = riccati(n, m, T, &W, alpha, NULL);
    if (!st) forward_pass(n, m, T, &W);
#define CP(dst, src, cnt) if (dst) memcpy(dst, src, sizeof(double) * (size_t)(cnt))
    CP(lam, W.lam, (T + 1) * n);
    CP(d, W.d, T * m);
    CP(S, W.S, (T + 1) * n * n);
    CP(s, W.s, (T + 1) * n);
    CP(Gam, W.Gam, T * m * n);
    CP(gam, W.gam, T * m);
    CP(dx, W.dx, (T + 1) * n);
    CP(du, W.du, T * m);
    CP(Pm, W.Pm, (T + 1) * n * n);
    CP(Mm, W.Mm, T * n * m);
    CP(Rm, W.Rm, T * m * m);
    CP(F, W.F, T * n * n);
    CP(Gm, W.G, T * n * m);
#undef CP
    if (g12) { g12[0] = W.G1; g12[1] = W.G2; }
    ws_free(&W);
    return st;
}

/* Public: one Newton direction of the multiplier form at (x, u) with multipliers nu
 * ((T+1) x n; row 0 is replaced by its local definition, see multiplier_pass).
 * Outputs (any may be NULL): q (T+1)xn, d Txm, dx (T+1)xn, du Txm, dnu (T+1)xn (the dual
 * step S_t dx_t + s_t), g12[2] = (G1, G2).  Returns 0, or 1 when R~ or Q is not positive
 * definite. */
int orc_newton_direction_mult(const orc_problem *P, const orc_aug *G, int T, const double *x,
                              const double *u, const double *nu_in, double alpha, double *q_out,
                              double *d, double *dx, double *du, double *dnu, double *g12)
{
    int n = P->nx, m = P->nu;
    rows_t R;
    build_rows(P, &R);
    newton_ws W;
    ws_alloc(&W, T, n, m);
    double *nu = malloc(sizeof(double) * (T + 1) * n), *q = calloc((size_t)(T + 1) * n, sizeof(double));
    memcpy(nu, nu_in, sizeof(double) * (T + 1) * n);
    multiplier_pass(P, &R, G, T, x, u, nu, &W, q);
    quadratize(P, &R, G, T, x, u, &W);
    int st = riccati(n, m, T, &W, alpha, q);
    if (!st) {
        forward_pass(n, m, T, &W);
        mult_g1(n, T, q, &W);
        if (dnu) mult_dual(n, T, &W, dnu);
    }
    if (q_out) memcpy(q_out, q, sizeof(double) * (T + 1) * n);
    if (d) memcpy(d, W.d, sizeof(double) * T * m);
    if (dx) memcpy(dx, W.dx, sizeof(double) * (T + 1) * n);
    if (du) memcpy(du, W.du, sizeof(double) * T * m);
    if (g12) { g12[0] = W.G1; g12[1] = W.G2; }
    free(nu);
    free(q);
    ws_free(&W);
    return st;
}

/* ------------------------------------------------------------------ */
/* associative elements and operators exactly as the paper defines them */
/* ------------------------------------------------------------------ */

/* Co-state operator (eq. co-states-comb-rule): element (j,t) then (t,i):
 *   g_{j,i} = g_{j,t} + F_{j,t}^T g_{t,i},   F^T_{j,i} = F^T_{j,t} F^T_{t,i}.
 * Ft arguments hold the transposed matrices F^T (n x n).  (The paper keeps dl/dx and
 * dc/dx as two vectors with the same rule; g is their sum.) */
void orc_costate_combine(int n, const double *g1, const double *Ft1, const double *g2,
                         const double *Ft2, double *g, double *Ft)
{
    double tg[ORC_MAXN], tF[ORC_MAXN * ORC_MAXN];
    for (int i = 0; i < n; i++) {
        double v = g1[i];
        for (int k = 0; k < n; k++) v += Ft1[i * n + k] * g2[k];
        tg[i] = v;
    }
    mm(n, n, n, Ft1, Ft2, tF);
    memcpy(g, tg, sizeof(double) * n);
    memcpy(Ft, tF, sizeof(double) * n * n);
}

/* Value-function element initialisation (eq. value-fun-elem-init) in the P^{-1}-free
 * form, which is algebraically identical to the printed one whenever P_t is invertible:
 *   A = F - G R~^{-1} M^T,  J = P - M R~^{-1} M^T,  C = G R~^{-1} G^T,
 *   eta = M R~^{-1} d,  b = -G R~^{-1} d.
 * reading: the printed form needs P_t^{-1}, which need not exist (P_t can be singular
 * or indefinite), so the equivalent form obtained by substituting q_t and r_t is used. */
int orc_value_init(int n, int m, const double *F, const double *Gm, const double *Pm,
                   const double *Mm, const double *Rm, const double *d, double alpha, double *A,
                   double *b, double *C, double *eta, double *J)
{
    double Rt[ORC_MAXM * ORC_MAXM], L[ORC_MAXM * ORC_MAXM], X[ORC_MAXM * (2 * ORC_MAXN + 1)];
    for (int i = 0; i < m * m; i++) Rt[i] = Rm[i];
    for (int i = 0; i < m; i++) Rt[i * m + i] += alpha;
    if (chol(m, Rt, L)) return 1;
    int c = 2 * n + 1;
    /* X = R~^{-1} [M^T | G^T | d] */
    for (int i = 0; i < m; i++) {
        for (int j = 0; j < n; j++) X[i * c + j] = Mm[j * m + i];
        for (int j = 0; j < n; j++) X[i * c + n + j] = Gm[j * m + i];
        X[i * c + 2 * n] = d[i];
    }
    chol_solve(m, c, L, X);
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            double gm = 0.0, mm_ = 0.0, gg = 0.0;
            for (int k = 0; k < m; k++) {
                gm += Gm[i * m + k] * X[k * c + j];
                mm_ += Mm[i * m + k] * X[k * c + j];
                gg += Gm[i * m + k] * X[k * c + n + j];
            }
            A[i * n + j] = F[i * n + j] - gm;
            J[i * n + j] = Pm[i * n + j] - mm_;
            C[i * n + j] = gg;
        }
        double e = 0.0, bb = 0.0;
        for (int k = 0; k < m; k++) {
            e += Mm[i * m + k] * X[k * c + 2 * n];
            bb += Gm[i * m + k] * X[k * c + 2 * n];
        }
        eta[i] = e;
        b[i] = -bb;
    }
    return 0;
}

/* The printed element initialisation (eq. value-fun-elem-init with q_t, r_t), which needs
 * P_t^{-1}; used only to pin the P^{-1}-free form.  Returns 1 if a matrix is singular. */
int orc_value_init_pinv(int n, int m, const double *F, const double *Gm, const double *Pm,
                        const double *Mm, const double *Rm, const double *d, double alpha,
                        double *A, double *b, double *C, double *eta, double *J)
{
    double Rt[ORC_MAXM * ORC_MAXM], PiM[ORC_MAXN * ORC_MAXM], S[ORC_MAXM * ORC_MAXM],
        q[ORC_MAXM], r[ORC_MAXN], X[ORC_MAXM * (2 * ORC_MAXN)], Y[ORC_MAXN * ORC_MAXN];
    for (int i = 0; i < m * m; i++) Rt[i] = Rm[i];
    for (int i = 0; i < m; i++) Rt[i * m + i] += alpha;
    memcpy(PiM, Mm, sizeof(double) * n * m);
    if (lu_solve(n, m, Pm, PiM)) return 1;          /* P^{-1} M */
    mtm(m, n, m, Mm, PiM, S);                       /* M^T P^{-1} M */
    for (int i = 0; i < m * m; i++) S[i] = Rt[i] - S[i];
    for (int i = 0; i < m; i++) q[i] = -d[i];
    if (lu_solve(m, 1, S, q)) return 1;             /* q = -[R~ - M^T P^{-1} M]^{-1} d */
    for (int i = 0; i < n; i++) {                   /* r = -P^{-1} M q */
        double v = 0.0;
        for (int k = 0; k < m; k++) v += PiM[i * m + k] * q[k];
        r[i] = -v;
    }
    int c = 2 * n;
    for (int i = 0; i < m; i++) {                   /* X = R~^{-1} [M^T | G^T] */
        for (int j = 0; j < n; j++) X[i * c + j] = Mm[j * m + i];
        for (int j = 0; j < n; j++) X[i * c + n + j] = Gm[j * m + i];
    }
    if (lu_solve(m, c, Rt, X)) return 1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double gm = 0.0, mm_ = 0.0, gg = 0.0;
            for (int k = 0; k < m; k++) {
                gm += Gm[i * m + k] * X[k * c + j];
                mm_ += Mm[i * m + k] * X[k * c + j];
                gg += Gm[i * m + k] * X[k * c + n + j];
            }
            A[i * n + j] = F[i * n + j] - gm;
            Y[i * n + j] = Pm[i * n + j] - mm_;
            C[i * n + j] = gg;
        }
    memcpy(J, Y, sizeof(double) * n * n);
    for (int i = 0; i < n; i++) {                   /* eta = [P - M R~^{-1} M^T] r */
        double v = 0.0;
        for (int k = 0; k < n; k++) v += Y[i * n + k] * r[k];
        eta[i] = v;
    }
    for (int i = 0; i < n; i++) {                   /* b = G R~^{-1} M^T r + G q */
        double v = 0.0;
        for (int k = 0; k < m; k++) {
            double w = q[k];
            for (int j = 0; j < n; j++) w += X[k * c + j] * r[j];
            v += Gm[i * m + k] * w;
        }
        b[i] = v;
    }
    return 0;
}

/* Value-function operator (eq. value-fun-param), element 1 = (j,t), element 2 = (t,i):
 *   A   = A2 (I + C1 J2)^{-1} A1
 *   J   = A1^T (I + J2 C1)^{-1} J2 A1 + J1
 *   C   = A2 (I + C1 J2)^{-1} C1 A2^T + C2
 *   eta = A1^T (I + J2 C1)^{-1} (eta2 - J2 b1) + eta1
 *   b   = A2 (I + C1 J2)^{-1} (b1 + C1 eta2) + b2
 * reading: the printed last line ends in "+ b_{j,i}", which makes the rule recursive;
 * the operator it is derived from adds b_{t,i} (b2).  Returns 1 if I + C1 J2 or
 * I + J2 C1 is singular. */
int orc_value_combine(int n, const double *A1, const double *b1, const double *C1,
                      const double *eta1, const double *J1, const double *A2, const double *b2,
                      const double *C2, const double *eta2, const double *J2, double *A,
                      double *b, double *C, double *eta, double *J)
{
    double M1[ORC_MAXN * ORC_MAXN], M2[ORC_MAXN * ORC_MAXN], T1[ORC_MAXN * ORC_MAXN];
    double X[ORC_MAXN * (2 * ORC_MAXN + 1)], Y[ORC_MAXN * (ORC_MAXN + 1)];
    double oA[ORC_MAXN * ORC_MAXN], oC[ORC_MAXN * ORC_MAXN], oJ[ORC_MAXN * ORC_MAXN],
        ob[ORC_MAXN], oe[ORC_MAXN], tmp[ORC_MAXN * ORC_MAXN], A2t[ORC_MAXN * ORC_MAXN];
    mm(n, n, n, C1, J2, T1);
    for (int i = 0; i < n * n; i++) M1[i] = T1[i];
    for (int i = 0; i < n; i++) M1[i * n + i] += 1.0;   /* I + C1 J2 */
    mm(n, n, n, J2, C1, T1);
    for (int i = 0; i < n * n; i++) M2[i] = T1[i];
    for (int i = 0; i < n; i++) M2[i * n + i] += 1.0;   /* I + J2 C1 */
    int c = 2 * n + 1;
    /* X = (I + C1 J2)^{-1} [A1 | C1 | b1 + C1 eta2] */
    for (int i = 0; i < n; i++) {
        double v = b1[i];
        for (int k = 0; k < n; k++) v += C1[i * n + k] * eta2[k];
        for (int j = 0; j < n; j++) { X[i * c + j] = A1[i * n + j]; X[i * c + n + j] = C1[i * n + j]; }
        X[i * c + 2 * n] = v;
    }
    if (lu_solve(n, c, M1, X)) return 1;
    /* Y = (I + J2 C1)^{-1} [J2 A1 | eta2 - J2 b1] */
    int cy = n + 1;
    mm(n, n, n, J2, A1, T1);
    for (int i = 0; i < n; i++) {
        double v = eta2[i];
        for (int k = 0; k < n; k++) v -= J2[i * n + k] * b1[k];
        for (int j = 0; j < n; j++) Y[i * cy + j] = T1[i * n + j];
        Y[i * cy + n] = v;
    }
    if (lu_solve(n, cy, M2, Y)) return 1;
    transpose(n, n, A2, A2t);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double a = 0.0, cc = 0.0;
            for (int k = 0; k < n; k++) {
                a += A2[i * n + k] * X[k * c + j];
                cc += A2[i * n + k] * X[k * c + n + j];
            }
            oA[i * n + j] = a;
            tmp[i * n + j] = cc;                       /* A2 (I+C1J2)^{-1} C1 */
        }
    mm(n, n, n, tmp, A2t, oC);
    for (int i = 0; i < n * n; i++) oC[i] += C2[i];
    for (int i = 0; i < n; i++) {
        double v = b2[i];
        for (int k = 0; k < n; k++) v += A2[i * n + k] * X[k * c + 2 * n];
        ob[i] = v;
    }
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            double v = J1[i * n + j];
            for (int k = 0; k < n; k++) v += A1[k * n + i] * Y[k * cy + j];
            oJ[i * n + j] = v;
        }
        double v = eta1[i];
        for (int k = 0; k < n; k++) v += A1[k * n + i] * Y[k * cy + n];
        oe[i] = v;
    }
    memcpy(A, oA, sizeof(double) * n * n);
    memcpy(C, oC, sizeof(double) * n * n);
    memcpy(J, oJ, sizeof(double) * n * n);
    memcpy(b, ob, sizeof(double) * n);
    memcpy(eta, oe, sizeof(double) * n);
    return 0;
}

/* State-propagation operator (eq. state-prop-comb-rule), element 1 = (j,t), 2 = (t,i):
 *   F_{j,i} = F_{t,i} F_{j,t},  e_{j,i} = F_{t,i} e_{j,t} + e_{t,i}. */
void orc_state_combine(int n, const double *F1, const double *e1, const double *F2,
                       const double *e2, double *F, double *e)
{
    double tF[ORC_MAXN * ORC_MAXN], te[ORC_MAXN];
    mm(n, n, n, F2, F1, tF);
    for (int i = 0; i < n; i++) {
        double v = e2[i];
        for (int k = 0; k < n; k++) v += F2[i * n + k] * e1[k];
        te[i] = v;
    }
    memcpy(F, tF, sizeof(double) * n * n);
    memcpy(e, te, sizeof(double) * n);
}

/* ------------------------------------------------------------------ */
/* step acceptance, Newton loop, IP and ADMM                            */
/* ------------------------------------------------------------------ */

/* Closed-loop nonlinear rollout for step size s (reading of Alg. 4's update, which as
 * printed leaves dynamics defects): u_t = u^_t + s gam_t + Gam_t (x_t - x^_t),
 * x_{t+1} = f(x_t, u_t), x_1 = x^_1.  Returns 1 if a value is not finite. */
static int rollout_closed(const orc_problem *P, int T, const double *xh, const double *uh,
                          const double *Gam, const double *gam, double s, double *x, double *u)
{
    int n = P->nx, m = P->nu;
    memcpy(x, xh, sizeof(double) * n);
    for (int t = 0; t < T; t++) {
        const double *xt = x + t * n, *xht = xh + t * n;
        double *ut = u + t * m;
        for (int i = 0; i < m; i++) {
            double v = uh[t * m + i] + s * gam[t * m + i];
            for (int j = 0; j < n; j++) v += Gam[(size_t)t * m * n + i * n + j] * (xt[j] - xht[j]);
            ut[i] = v;
        }
        orc_step(P, xt, ut, x + (t + 1) * n);
        for (int i = 0; i < n; i++)
            if (!isfinite(x[(t + 1) * n + i])) return 1;
    }
    return 0;
}

typedef struct { int iters, ls_rejects, factor_fails; double alpha; } nstats;

/* Newton iterations (Alg. 4) on the augmented sub-problem eq. augmented-ocp until
 * max_t |d_t|_inf <= tol.  Step acceptance (reading; the paper gives no rule): candidate
 * steps s = 1, beta, beta^2, ... (ls_count of them); accept the largest s whose rollout
 * is finite, strictly feasible for the barrier, and satisfies
 *   J_c(s) <= J_c(0) + c1 s G1 + eps (1 + |J_c(0)|).
 * Regularisation (reading of "(2.21) of Madsen et al." cited in Sec. III-E): gain ratio
 * rho = (J_c(0) - J_c(s)) / -(s G1 + s^2 G2); rho > 0.75 -> alpha /= 3, rho < 0.25 ->
 * alpha *= 2, clamped to [alpha_min, alpha_max]; a failed factorisation sets
 * alpha = max(10 alpha, 1e-8) and retries; no accepted step multiplies alpha by 10. */
static int newton_solve(const orc_problem *P, const rows_t *R, const orc_aug *G,
                        const orc_options *o, int T, double *x, double *u, double tol,
                        nstats *st, double *rfinal, double *nu)
{
    int n = P->nx, m = P->nu, rc = ORC_ENOTCONV;
    newton_ws W;
    ws_alloc(&W, T, n, m);
    double *xc = malloc(sizeof(double) * (T + 1) * n), *uc = malloc(sizeof(double) * (T * m + 1));
    double *q = nu ? calloc((size_t)(T + 1) * n, sizeof(double)) : NULL;
    if (nu && o->costate_mode == 2) {
        /* hybrid: each sub-problem (barrier level, ADMM iteration) starts from the
         * co-states of the recursion; multiplier steps take over from there */
        costate_pass(P, R, G, T, x, u, &W);
        memcpy(nu, W.lam, sizeof(double) * (T + 1) * n);
    }
    double J0 = traj_cost(P, R, G, T, x, u, NULL);
    double r = INFINITY;
    for (int it = 0; it <= o->max_newton; it++) {
        r = nu ? multiplier_pass(P, R, G, T, x, u, nu, &W, q) : costate_pass(P, R, G, T, x, u, &W);
        if (r <= tol) { rc = ORC_OK; break; }
        if (it == o->max_newton || !isfinite(r) || !isfinite(J0)) break;
        st->iters++;
        quadratize(P, R, G, T, x, u, &W);
        while (riccati(n, m, T, &W, st->alpha, q)) {
            st->factor_fails++;
            st->alpha = fmax(10.0 * st->alpha, 1e-8);
            if (st->alpha > o->alpha_max) { rc = ORC_ENUM; goto done; }
        }
        forward_pass(n, m, T, &W);
        if (q) mult_g1(n, T, q, &W);
        int accepted = 0;
        double s = 1.0, Js = INFINITY;
        if (o->update_mode == 1) {
            /* Alg. 4 as printed: the full Newton step on states and controls, no rollout
             * (the linearised dynamics leave defects x_{t+1} - f(x_t, u_t) of second order).
             * Reading: the step is taken whenever its cost is finite (for the barrier: the
             * point is strictly feasible); otherwise it counts as rejected. */
            for (int i = 0; i < (T + 1) * n; i++) xc[i] = x[i] + W.dx[i];
            for (int i = 0; i < T * m; i++) uc[i] = u[i] + W.du[i];
            Js = traj_cost(P, R, G, T, xc, uc, NULL);
            accepted = isfinite(Js);
        } else {
            for (int k = 0; k < o->ls_count; k++, s *= o->ls_beta) {
                if (rollout_closed(P, T, x, u, W.Gam, W.gam, s, xc, uc)) continue;
                Js = traj_cost(P, R, G, T, xc, uc, NULL);
                if (!isfinite(Js)) continue;
                if (Js <= J0 + o->armijo_c1 * s * W.G1 + o->armijo_eps * (1.0 + fabs(J0))) {
                    accepted = 1;
                    break;
                }
            }
        }
        if (accepted) {
            double pred = -(s * W.G1 + s * s * W.G2);
            double rho = pred > 0.0 ? (J0 - Js) / pred : 0.0;
            if (rho > 0.75) st->alpha /= 3.0;
            else if (rho < 0.25) st->alpha *= 2.0;
            st->alpha = fmin(fmax(st->alpha, o->alpha_min), o->alpha_max);
            memcpy(x, xc, sizeof(double) * (T + 1) * n);
            memcpy(u, uc, sizeof(double) * T * m);
            J0 = Js;
            if (nu) {
                /* multipliers := the duals of the LQR's linearised dynamics, nu + dnu
                 * (the full dual step whatever the primal step s: the LQR duals are the
                 * multiplier estimate at the linearisation point) */
                mult_dual(n, T, &W, q);
                for (int i = 0; i < (T + 1) * n; i++) nu[i] += q[i];
            }
        } else {
            st->ls_rejects++;
            st->alpha *= 10.0;
            if (st->alpha > o->alpha_max) { rc = ORC_ENUM; break; }
        }
    }
done:
    if (rfinal) *rfinal = r;
    free(xc);
    free(uc);
    free(q);
    ws_free(&W);
    return rc;
}

/* info layout (16 doubles):
 *  0 status  1 newton iterations  2 outer iterations  3 mu  4 alpha  5 r_stat  6 r_dyn
 *  7 r_feas  8 r_kkt  9 J  10 J_c  11 r_p  12 r_d  13 line-search rejects  14 factor fails */
static void residuals(const orc_problem *P, const rows_t *R, const orc_aug *G, int T,
                      const double *x, const double *u, double *lam_out, double *info,
                      double *nu)
{
    int n = P->nx, m = P->nu;
    newton_ws W;
    ws_alloc(&W, T, n, m);
    double *q = nu ? calloc((size_t)(T + 1) * n, sizeof(double)) : NULL;
    /* multiplier form: stationarity of the Lagrangian in u and x (both gradients), and
     * the multipliers as the co-states */
    double rs = nu ? multiplier_pass(P, R, G, T, x, u, nu, &W, q) : costate_pass(P, R, G, T, x, u, &W);
    free(q);
    double rd = 0.0, rf = 0.0, xn[ORC_MAXN];
    for (int t = 0; t < T; t++) {
        orc_step(P, x + t * n, u + t * m, xn);
        for (int i = 0; i < n; i++) rd = fmax(rd, fabs(x[(t + 1) * n + i] - xn[i]));
        for (int r = 0; r < R->nw; r++) rf = fmax(rf, row_value(R, r, x + t * n, u + t * m));
        if (P->ucons && P->nc > 0) {
            double g[ORC_MAXC];
            P->ucons(P->uctx, t, x + t * n, u + t * m, g, NULL, NULL);
            for (int c = 0; c < P->nc; c++) rf = fmax(rf, g[c]);
        }
    }
    double Jp;
    double Jc = traj_cost(P, R, G, T, x, u, &Jp);
    if (!isfinite(Jc)) {
        orc_aug none = {AUG_NONE, 0, 0.0, 0.0, NULL, NULL};
        traj_cost(P, R, &none, T, x, u, &Jp);
    }
    info[5] = rs;
    info[6] = rd;
    info[7] = fmax(rf, 0.0);
    info[9] = Jp;
    info[10] = Jc;
    if (lam_out) memcpy(lam_out, W.lam, sizeof(double) * (T + 1) * n);
    ws_free(&W);
}

static int check_feasible(const orc_problem *P, const rows_t *R, int T, const double *x,
                          const double *u)
{
    int n = P->nx, m = P->nu;
    for (int t = 0; t < T; t++) {
        for (int r = 0; r < R->nw; r++)
            if (!(row_value(R, r, x + t * n, u + t * m) < 0.0)) return 0;
        if (P->ucons && P->nc > 0) {
            double g[ORC_MAXC];
            P->ucons(P->uctx, t, x + t * n, u + t * m, g, NULL, NULL);
            for (int c = 0; c < P->nc; c++)
                if (!(g[c] < 0.0)) return 0;
        }
    }
    return 1;
}

/* Primal log-barrier IP (Sec. II-B, eq. lb-min, lb-step-2): mu_k = mu0 zeta^k, each barrier
 * sub-problem solved by Newton (Alg. 4) warm-started from the previous result, until the
 * level mu <= mu_final has been solved.  reading: inner tolerance tol_inner for
 * mu > mu_final and tol_final at mu_final (the paper gives no value). */
int orc_solve_ip(const orc_problem *P, const orc_options *o, const double *x0,
                 const double *u_init, int T, double *x, double *u, double *lam, double *info)
{
    int n = P->nx, m = P->nu;
    memset(info, 0, sizeof(double) * 16);
    if (T < 1 || n < 1 || n > ORC_MAXN || m < 1 || m > ORC_MAXM) { info[0] = ORC_EINVAL; return ORC_EINVAL; }
    rows_t R;
    build_rows(P, &R);
    if (u_init) memcpy(u, u_init, sizeof(double) * T * m);
    else memset(u, 0, sizeof(double) * T * m);
    orc_rollout(P, x0, u, T, x);
    if (!check_feasible(P, &R, T, x, u)) { info[0] = ORC_EINFEAS; return ORC_EINFEAS; }
    nstats st = {0, 0, 0, o->alpha0};
    /* multiplier form: nu starts at zero (no recursion through F^T at the start either) */
    double *nu = o->costate_mode != 0 ? calloc((size_t)(T + 1) * n, sizeof(double)) : NULL;
    double mu = o->mu0;
    int rc = ORC_OK, level = 0;
    orc_aug G = {AUG_BARRIER, R.nw, mu, 0.0, NULL, NULL};
    for (;;) {
        int last = mu <= o->mu_final * (1.0 + 1e-9);
        G.mu = mu;
        rc = newton_solve(P, &R, &G, o, T, x, u, last ? o->tol_final : o->tol_inner, &st, NULL, nu);
        level++;
        if (rc == ORC_ENUM || last) break;
        mu = o->mu0 * pow(o->zeta, level);
        if (mu < o->mu_final) mu = o->mu_final;
    }
    residuals(P, &R, &G, T, x, u, lam, info, nu);
    free(nu);
    info[0] = rc;
    info[1] = st.iters;
    info[2] = level;
    info[3] = mu;
    info[4] = st.alpha;
    info[8] = fmax(fmax(info[5], info[6]), fmax(info[7], mu));
    info[13] = st.ls_rejects;
    info[14] = st.factor_fails;
    return rc;
}

/* Newton on the barrier problem at one fixed mu (warm start from u_init); used by the
 * finite-difference checks of the adjoint. */
int orc_solve_fixed_mu(const orc_problem *P, const orc_options *o, double mu, double tol,
                       const double *x0, const double *u_init, int T, double *x, double *u,
                       double *lam, double *info)
{
    int m = P->nu;
    memset(info, 0, sizeof(double) * 16);
    rows_t R;
    build_rows(P, &R);
    memcpy(u, u_init, sizeof(double) * T * m);
    orc_rollout(P, x0, u, T, x);
    if (!check_feasible(P, &R, T, x, u)) { info[0] = ORC_EINFEAS; return ORC_EINFEAS; }
    nstats st = {0, 0, 0, o->alpha0};
    orc_aug G = {AUG_BARRIER, R.nw, mu, 0.0, NULL, NULL};
    double *nu = o->costate_mode != 0 ? calloc((size_t)(T + 1) * P->nx, sizeof(double)) : NULL;
    int rc = newton_solve(P, &R, &G, o, T, x, u, tol, &st, NULL, nu);
    residuals(P, &R, &G, T, x, u, lam, info, nu);
    free(nu);
    info[0] = rc;
    info[1] = st.iters;
    info[3] = mu;
    info[4] = st.alpha;
    return rc;
}

/* ADMM (Sec. II-C, eq. admm-min ... admm-step-5) with w = [g; h] stacked per step.
 * z and v (T x nw, may be NULL) receive the final consensus variables and multipliers.
 * reading: the
 * v-update uses w(x, u) where the paper prints y_t; z^0 = min(0, w(x^0, u^0)), v^0 = 0;
 * r_d = z^k - z^{k-1} without a rho factor, as printed.  When fixed_iters > 0 exactly
 * that many outer iterations run (for comparisons at a fixed outer count). */
int orc_solve_admm(const orc_problem *P, const orc_options *o, const double *x0,
                   const double *u_init, int T, double *z, double *v, double *x, double *u,
                   double *lam, double *info)
{
    int n = P->nx, m = P->nu;
    memset(info, 0, sizeof(double) * 16);
    if (T < 1 || n < 1 || n > ORC_MAXN || m < 1 || m > ORC_MAXM) { info[0] = ORC_EINVAL; return ORC_EINVAL; }
    if (P->ucons && P->nc > 0) { info[0] = ORC_EINVAL; return ORC_EINVAL; }  /* user rows: IP only */
    rows_t R;
    build_rows(P, &R);
    int nw = R.nw;
    if (u_init) memcpy(u, u_init, sizeof(double) * T * m);
    else memset(u, 0, sizeof(double) * T * m);
    orc_rollout(P, x0, u, T, x);
    double *zi = malloc(sizeof(double) * ((size_t)T * nw + 1)), *vi = malloc(sizeof(double) * ((size_t)T * nw + 1));
    double *zp = malloc(sizeof(double) * ((size_t)T * nw + 1));
    for (int t = 0; t < T; t++)
        for (int r = 0; r < nw; r++) {
            double w = row_value(&R, r, x + t * n, u + t * m);
            zi[t * nw + r] = w < 0.0 ? w : 0.0;
            vi[t * nw + r] = 0.0;
        }
    nstats st = {0, 0, 0, o->alpha0};
    double *nu = o->costate_mode != 0 ? calloc((size_t)(T + 1) * n, sizeof(double)) : NULL;
    orc_aug G = {AUG_ADMM, nw, 0.0, o->rho, zi, vi};
    int rc = ORC_ENOTCONV, k;
    double rp = INFINITY, rdl = INFINITY;
    int kmax = o->admm_fixed_iters > 0 ? o->admm_fixed_iters : o->max_outer;
    for (k = 0; k < kmax; k++) {
        int s = newton_solve(P, &R, &G, o, T, x, u, o->tol_final, &st, NULL, nu);
        if (s == ORC_ENUM) { rc = ORC_ENUM; k++; break; }
        memcpy(zp, zi, sizeof(double) * T * nw);
        rp = 0.0;
        rdl = 0.0;
        for (int t = 0; t < T; t++)
            for (int r = 0; r < nw; r++) {
                double w = row_value(&R, r, x + t * n, u + t * m);
                double zn = w + vi[t * nw + r] / o->rho;
                zn = zn < 0.0 ? zn : 0.0;                    /* projection onto w <= 0 */
                vi[t * nw + r] += o->rho * (w - zn);
                zi[t * nw + r] = zn;
                rp = fmax(rp, fabs(w - zn));
                rdl = fmax(rdl, fabs(zn - zp[t * nw + r]));
            }
        if (o->admm_fixed_iters <= 0 && rp <= o->admm_tol && rdl <= o->admm_tol) { rc = ORC_OK; k++; break; }
    }
    if (o->admm_fixed_iters > 0 && rc != ORC_ENUM) rc = ORC_OK;
    residuals(P, &R, &G, T, x, u, lam, info, nu);
    free(nu);
    info[0] = rc;
    info[1] = st.iters;
    info[2] = k;
    info[4] = st.alpha;
    info[11] = rp;
    info[12] = rdl;
    info[13] = st.ls_rejects;
    info[14] = st.factor_fails;
    if (z) memcpy(z, zi, sizeof(double) * T * nw);
    if (v) memcpy(v, vi, sizeof(double) * T * nw);
    free(zi);
    free(vi);
    free(zp);
    return rc;
}

/* ------------------------------------------------------------------ */
/* adjoint                                                             */
/* ------------------------------------------------------------------ */

/* Gradients of a scalar loss  L = gJ * J*  +  sum gx . x*  +  sum gu . u*  at a solution
 * (x*, u*) of the barrier problem at barrier weight mu, with respect to
 *   x0 (n), diag Q (n), diag R (m), diag Qf (n), and the model constants prm (ORC_MAXP).
 * J* part (J* = optimal barrier objective, written Jopt): envelope theorem on the Lagrangian eq. ocp-lagrangian (dJopt/dx0 = lam_1,
 *   dJopt/dtheta = dL_c/dtheta).
 * x*, u* part: implicit function theorem on the KKT system; the adjoint LQR
 *   min 1/2 w^T H w - g^T w  s.t. w_{x,t+1} = F w_{x,t} + G w_{u,t}, w_{x,1} = 0
 *   (H = the Newton-step Hessian with alpha = 0) is solved by the Riccati recursion, its
 *   multipliers nu by the co-state recursion nu_t = P w_x + M w_u - gx_t + F^T nu_{t+1},
 *   and dL/dtheta = -w^T d_theta(grad_z L) - nu^T d_theta(constraints).
 * Returns 0, or 1 if the Hessian is not positive definite at the solution. */
int orc_adjoint(const orc_problem *P, double mu, int T, const double *x, const double *u,
                double gJ, const double *gx, const double *gu, double *g_x0, double *g_Qd,
                double *g_Rd, double *g_Qfd, double *g_prm)
{
    int n = P->nx, m = P->nu;
    rows_t R;
    build_rows(P, &R);
    orc_aug G = {AUG_BARRIER, R.nw, mu, 0.0, NULL, NULL};
    newton_ws W;
    ws_alloc(&W, T, n, m);
    costate_pass(P, &R, &G, T, x, u, &W);
    double dfdp[ORC_MAXN * ORC_MAXP], Hzp[(ORC_MAXN + ORC_MAXM) * ORC_MAXP];
    for (int i = 0; i < n; i++) {
        g_x0[i] = gJ * W.lam[i];
        double sq = 0.0;
        for (int t = 0; t < T; t++) { double e = x[t * n + i] - xref_at(P, t)[i]; sq += e * e; }
        g_Qd[i] = P->ustage ? 0.0 : gJ * sq;  /* a user stage cost does not depend on Q, R */
        double e = x[T * n + i] - xref_at(P, T)[i];
        g_Qfd[i] = P->uterm ? 0.0 : gJ * e * e;
    }
    for (int i = 0; i < m; i++) {
        double sq = 0.0;
        for (int t = 0; t < T; t++) { double e = u[t * m + i] - uref_at(P, t)[i]; sq += e * e; }
        g_Rd[i] = P->ustage ? 0.0 : gJ * sq;
    }
    for (int k = 0; k < ORC_MAXP; k++) g_prm[k] = 0.0;
    for (int t = 0; t < T; t++) {
        orc_param_jac(P, x + t * n, u + t * m, dfdp);
        for (int k = 0; k < ORC_MAXP; k++) {
            double v = 0.0;
            for (int i = 0; i < n; i++) v += W.lam[(t + 1) * n + i] * dfdp[i * ORC_MAXP + k];
            g_prm[k] += gJ * v;
        }
    }
    int rc = 0;
    if (gx || gu) {
        quadratize(P, &R, &G, T, x, u, &W);
        double *qx = calloc((size_t)(T + 1) * n, sizeof(double));
        for (int i = 0; i < (T + 1) * n; i++) qx[i] = gx ? -gx[i] : 0.0;
        for (int i = 0; i < T * m; i++) W.d[i] = gu ? -gu[i] : 0.0;
        if (riccati(n, m, T, &W, 0.0, qx)) { rc = 1; free(qx); goto out; }
        forward_pass(n, m, T, &W);               /* W.dx = w_x, W.du = w_u */
        double *nu = calloc((size_t)(T + 1) * n, sizeof(double));
        const double *PT = W.Pm + (size_t)T * n * n;
        for (int i = 0; i < n; i++) {
            double v = qx[T * n + i];
            for (int j = 0; j < n; j++) v += PT[i * n + j] * W.dx[T * n + j];
            nu[T * n + i] = v;
        }
        for (int t = T - 1; t >= 0; t--) {
            const double *F = W.F + (size_t)t * n * n, *Pt = W.Pm + (size_t)t * n * n,
                         *Mt = W.Mm + (size_t)t * n * m;
            for (int i = 0; i < n; i++) {
                double v = qx[t * n + i];
                for (int j = 0; j < n; j++) v += Pt[i * n + j] * W.dx[t * n + j] + F[j * n + i] * nu[(t + 1) * n + j];
                for (int j = 0; j < m; j++) v += Mt[i * m + j] * W.du[t * m + j];
                nu[t * n + i] = v;
            }
        }
        for (int i = 0; i < n; i++) {
            g_x0[i] -= nu[i];
            double a = 0.0;
            for (int t = 0; t < T; t++) a += W.dx[t * n + i] * 2.0 * (x[t * n + i] - xref_at(P, t)[i]);
            if (!P->ustage) g_Qd[i] -= a;
            if (!P->uterm) g_Qfd[i] -= W.dx[T * n + i] * 2.0 * (x[T * n + i] - xref_at(P, T)[i]);
        }
        for (int i = 0; i < m; i++) {
            double a = 0.0;
            for (int t = 0; t < T; t++) a += W.du[t * m + i] * 2.0 * (u[t * m + i] - uref_at(P, t)[i]);
            if (!P->ustage) g_Rd[i] -= a;
        }
        for (int t = 0; t < T; t++) {
            orc_param_jac(P, x + t * n, u + t * m, dfdp);
            orc_param_hess(P, x + t * n, u + t * m, W.lam + (t + 1) * n, Hzp);
            for (int k = 0; k < ORC_MAXP; k++) {
                double v = 0.0;
                for (int j = 0; j < n; j++) v += W.dx[t * n + j] * Hzp[j * ORC_MAXP + k];
                for (int j = 0; j < m; j++) v += W.du[t * m + j] * Hzp[(n + j) * ORC_MAXP + k];
                for (int i = 0; i < n; i++) v += nu[(t + 1) * n + i] * dfdp[i * ORC_MAXP + k];
                g_prm[k] -= v;
            }
        }
        free(nu);
        free(qx);
    }
out:
    ws_free(&W);
    return rc;
}
