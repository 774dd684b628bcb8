/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the phase-field lattice Boltzmann
 * method of "Freezing dynamics of wetting droplet under a uniform electric
 * field" (Huang, Li, Che, Chai, Wang, Shi; arXiv 2410.06657).
 *
 * TEST INFRASTRUCTURE ONLY.  This code defines what "correct" means for the
 * GPU library.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the library never calls it.  It shares no
 * source, header, table or helper with the CUDA code.
 *
 * Style: plain loops, double precision, one field at a time, in the order the
 * paper's Algorithm 1 names the steps, with no blocking or fusion.  Build it
 * with -ffp-contract=off so every product and sum is rounded as written.
 *
 * Where the paper is silent or garbled, the following readings are taken
 * (each one is cited again where it is used):
 *   R1  All four systems collide with time-n macroscopic fields (a Jacobi
 *       split of Algorithm 1's sequence); then all stream; then boundaries.
 *   R2  n = grad(psi)/|grad(psi)| and kappa*lap(psi) (Sec. 2 prints phi).
 *       Sec. 2 leaves n undefined where grad(psi) vanishes; the normal is
 *       regularised as grad(psi) / (|grad(psi)| + 1e-4).  Without it, cells
 *       whose psi sits slightly off 0 or 1 (lambda = 4 psi (1 - psi)/W not
 *       small) but whose gradient is at round-off level get a counter-flux
 *       M lambda n of fixed size in a direction set by round-off, which
 *       amplifies last-bit differences by ~1e8 within 200 steps.
 *   R5  H_s = C_p T_m, T_s = T_l = T_m (pure substance).
 *   R6  Latent heat is carried by the liquid only: L_eff = psi L,
 *       f_l = clamp((H - H_s)/L_eff, 0, 1) (f_l = 1 where L_eff < 1e-12),
 *       f_s = psi (1 - f_l).  C_p in the inversion uses the lagged f_s.
 *   R7  psi and H recovery use the lagged mdot and Q = rho C_p T mdot.
 *   R8  div u := mdot (Eq. ns1).
 *   R9  "c_s^2 div S" read as c_s^2 grad S; grad p and grad S use the
 *       previous step's p and S.
 *   R10 "tau dt R_0" in Eq. (Computed_p) uses the local tau_h.
 *   R11 u_s = 0 (ice and substrate at rest): rho f = -rho f_s u*.
 *   R13 Enthalpy source weighted by w_i, prefactor (1 - 1/(2 tau_g)),
 *       tau_g = k/(rho C_p,ref c_s^2) + 1/2.
 *   R15 The potential is swept k_e times per step (sigma frozen at time n).
 *   R16 sigma_g sets tau_l in the gas; only the ratio R matters physically.
 *   R17 Wetting: ghost psi(-1) = psi(0) + (4/W) cos(theta) psi(0)(1-psi(0));
 *       top wall neutral (ghost = copy).
 *   R18 Dirichlet walls by half-way anti-bounce-back: g at the cold bottom
 *       wall (T_w), l at both electrodes; g at the top wall bounces back
 *       (adiabatic).  f and h bounce back at both walls.
 *   R19 Stencil ghosts: rho, eps, p, S copied; phi mirrored about phi_wall.
 *   R20 phi = 0 at the bottom electrode, E0 * ny at the top one,
 *       E0 = sqrt(CaE gamma / (eps_g R0)).
 *   R21 Solid mu, eps, sigma equal the liquid's; F_b = 0.  The solid's
 *       thermal diffusivity is alpha_l * alpha_sl (alpha_sl = 1 unless a
 *       property set such as Table 1 gives the solid its own).
 *   R24 Substrate heat flux (Sec. 4.3): Fourier's law with the one-sided
 *       second-order difference applied to the first three cell rows,
 *       Qdot(x) = -k(x,0) (4 T(x,1) - T(x,2) - 3 T(x,0)) / 2, k the local
 *       conductivity of row 0; the sign is the paper's (negative when heat
 *       flows into the cold wall).  Qdot in the observables is its sum over x.
 *   R25 Peclet number (Sec. 4.3): Pe = D_d u_d / alpha_l with D_d = 2 R0 and
 *       u_d the liquid-weighted mean speed, sum w |psi u| / psi over sum w,
 *       w = psi - f_s (the liquid content of a cell), using the psi u that
 *       the last step stored (the velocity at that step's start).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Problem parameters (dimensionless set plus lattice choices).        */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny;     /* lattice size; x periodic, walls at y=-1/2, ny-1/2 */
    int32_t k_e;        /* potential sweeps per time step (>= 1)             */
    int32_t reserved;
    double W;           /* interface width                                   */
    double M;           /* phase-field mobility                              */
    double gamma;       /* liquid-gas surface tension                        */
    double rho_l;       /* liquid density                                    */
    double rho_lg;      /* rho_l / rho_g                                     */
    double rho_sl;      /* rho_s / rho_l                                     */
    double mu_l;        /* liquid dynamic viscosity                          */
    double mu_lg;       /* mu_l / mu_g                                       */
    double Ste;         /* Stefan number C_p,l (T_m - T_w) / L               */
    double alpha_l;     /* liquid thermal diffusivity                        */
    double alpha_lg;    /* alpha_l / alpha_g                                 */
    double cp_l, cp_s, cp_g;
    double T_m, T_w, T_init;
    double CaE;         /* electric capillary number eps_g E0^2 R0 / gamma    */
    double R_sigma;     /* sigma_l / sigma_g                                 */
    double S_eps;       /* eps_l / eps_g                                     */
    double eps_g;       /* gas permittivity                                  */
    double sigma_g;     /* gas conductivity                                  */
    double R0;          /* reference radius (CaE, Fo)                        */
    double theta_deg;   /* static contact angle on the bottom wall           */
    double alpha_sl;    /* alpha_s / alpha_l (R21)                           */
} orc_params;

/* Phase-resolved properties in lattice units: index 0 solid, 1 liquid, 2 gas */
typedef struct {
    double rho[3], mu[3], kth[3], cp[3], eps[3], sig[3];
    double L, Cref, kappa, beta, tau_f, E0, phi_bot, phi_top, wet, alpha_s;
} orc_derived;

typedef struct {
    int64_t step;
    double Fo, mass, enthalpy, charge, solid, frozen_fraction;
    double height, width, aspect, R_tr, front;
    int64_t t_fre;
    double Fo_fre;
    int32_t status;
    int32_t reserved;
    double Pe;          /* R25 */
    double Qdot;        /* R24: sum over the substrate */
} orc_obs;

typedef struct {
    orc_params P;
    orc_derived D;
    int nx, ny;
    long N;
    int64_t step;
    int64_t t_fre;
    double *f, *h, *g, *l;          /* populations [q][y][x] at time n       */
    double *fs_prev, *mdot_prev, *Q_prev, *psiux_prev, *psiuy_prev;
    double *p_prev, *S_prev;        /* previous step's p and S (R9)          */
    double *sigma_n;                /* sigma used by the extra sweeps (R15)  */
} orc_state;

/* ------------------------------------------------------------------ */
/* Lattices (Sec. 3.1 D2Q9, Sec. 3.4 D2Q5).                             */
/* ------------------------------------------------------------------ */
static int CX[9], CY[9], OPP[9];
static double W9[9];
static const int CX5[5] = {0, 1, 0, -1, 0};     /* Sec. 3.4 matrix      */
static const int CY5[5] = {0, 0, 1, 0, -1};
static const int OPP5[5] = {0, 3, 4, 1, 2};
static const double W5[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
static const double CS2 = 1.0 / 3.0;            /* c_s = c / sqrt(3)    */
static int lattice_ready = 0;

/* c_i from the paper's cos/sin definition, rounded to the integer grid. */
static void build_lattice(void)
{
    if (lattice_ready) return;
    const double pi = 3.14159265358979323846;
    CX[0] = 0; CY[0] = 0; W9[0] = 4.0 / 9.0;
    for (int i = 1; i <= 4; i++) {
        CX[i] = (int)lround(cos((i - 1) * pi / 2.0));
        CY[i] = (int)lround(sin((i - 1) * pi / 2.0));
        W9[i] = 1.0 / 9.0;
    }
    for (int i = 5; i <= 8; i++) {
        CX[i] = (int)lround(sqrt(2.0) * cos((2 * i - 9) * pi / 4.0));
        CY[i] = (int)lround(sqrt(2.0) * sin((2 * i - 9) * pi / 4.0));
        W9[i] = 1.0 / 36.0;
    }
    for (int i = 0; i < 9; i++)
        for (int j = 0; j < 9; j++)
            if (CX[j] == -CX[i] && CY[j] == -CY[i]) OPP[i] = j;
    lattice_ready = 1;
}

/* Exported for the test suite: the D2Q9 table as this file derives it. */
void orc_lattice(int32_t *cx, int32_t *cy, double *w)
{
    build_lattice();
    for (int i = 0; i < 9; i++) { cx[i] = CX[i]; cy[i] = CY[i]; w[i] = W9[i]; }
}

/* ------------------------------------------------------------------ */
/* Derived lattice constants (Sec. 2 and the readings R16, R20-R21).    */
/* ------------------------------------------------------------------ */
int orc_derive(const orc_params *P, orc_derived *D)
{
    if (P->nx <= 0 || P->ny <= 0 || P->k_e < 1) return -1;
    if (!(P->W > 0) || !(P->M > 0) || !(P->gamma >= 0) || !(P->rho_l > 0) ||
        !(P->rho_lg > 0) || !(P->rho_sl > 0) || !(P->mu_l > 0) || !(P->mu_lg > 0) ||
        !(P->Ste > 0) || !(P->alpha_l > 0) || !(P->alpha_lg > 0) || !(P->cp_l > 0) ||
        !(P->cp_s > 0) || !(P->cp_g > 0) || !(P->CaE >= 0) || !(P->R_sigma > 0) ||
        !(P->S_eps > 0) || !(P->eps_g > 0) || !(P->sigma_g > 0) || !(P->R0 > 0) ||
        !(P->theta_deg > 0 && P->theta_deg < 180) || !(P->alpha_sl > 0))
        return -1;
    D->rho[1] = P->rho_l;
    D->rho[2] = P->rho_l / P->rho_lg;
    D->rho[0] = P->rho_l * P->rho_sl;
    D->mu[1] = P->mu_l;
    D->mu[2] = P->mu_l / P->mu_lg;
    D->mu[0] = P->mu_l;                                   /* R21 */
    D->cp[0] = P->cp_s; D->cp[1] = P->cp_l; D->cp[2] = P->cp_g;
    D->alpha_s = P->alpha_l * P->alpha_sl;                /* R21 */
    D->kth[1] = D->rho[1] * D->cp[1] * P->alpha_l;        /* k = rho C_p alpha */
    D->kth[2] = D->rho[2] * D->cp[2] * (P->alpha_l / P->alpha_lg);
    D->kth[0] = D->rho[0] * D->cp[0] * D->alpha_s;
    D->eps[2] = P->eps_g;
    D->eps[1] = P->S_eps * P->eps_g;                      /* S = eps_i/eps_e */
    D->eps[0] = D->eps[1];
    D->sig[2] = P->sigma_g;
    D->sig[1] = P->R_sigma * P->sigma_g;                  /* R = sigma_i/sigma_e */
    D->sig[0] = D->sig[1];
    D->L = P->cp_l * (P->T_m - P->T_w) / P->Ste;          /* Ste = C_p dT / L */
    D->Cref = 2.0 * P->cp_s * P->cp_l / (P->cp_s + P->cp_l);
    D->kappa = 1.5 * P->gamma * P->W;                     /* kappa = 3 gamma W / 2 */
    D->beta = 12.0 * P->gamma / P->W;
    D->tau_f = P->M / CS2 + 0.5;
    D->E0 = sqrt(P->CaE * P->gamma / (P->eps_g * P->R0)); /* CaE = eps_e E0^2 R/gamma */
    D->phi_bot = 0.0;                                     /* R20 */
    D->phi_top = D->E0 * P->ny;
    D->wet = 4.0 / P->W * cos(P->theta_deg * 3.14159265358979323846 / 180.0);
    if (!(D->L >= 0)) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Pointwise pieces of the scheme.                                      */
/* ------------------------------------------------------------------ */

/* Eq. (Computed): chi = f_s chi_s + (1-f_s) psi chi_l + (1-f_s)(1-psi) chi_g */
static double chi(double fs, double psi, const double v[3])
{
    return fs * v[0] + (1.0 - fs) * psi * v[1] + (1.0 - fs) * (1.0 - psi) * v[2];
}

/* Eq. (Hfl) with readings R5, R6: total enthalpy -> liquid fraction, T. */
void orc_enthalpy_inversion(double H, double psi, double cp, double Tm, double L,
                            double *fl, double *T)
{
    double Hs = cp * Tm;
    double Leff = psi * L;
    double Hl = Hs + Leff;
    if (H < Hs)
        *T = H / cp;
    else if (H <= Hl)
        *T = Tm;
    else
        *T = Tm + (H - Hl) / cp;
    if (Leff < 1e-12) {
        *fl = 1.0;
    } else {
        double r = (H - Hs) / Leff;
        *fl = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
    }
}

/* s_i(u) of Sec. 3.2 */
static double s_i(int i, double ux, double uy)
{
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return W9[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Sec. 3.1: phase-field equilibrium and source. */
static double f_eq(int i, double psi, double ux, double uy)
{
    double cu = CX[i] * ux + CY[i] * uy;
    return W9[i] * psi * (1.0 + cu / CS2);
}

static double f_src(int i, double psi, double dtx, double dty, double lam,
                    double nxv, double nyv, double divu)
{
    double ax = dtx + CS2 * lam * nxv;
    double ay = dty + CS2 * lam * nyv;
    return W9[i] * (CX[i] * ax + CY[i] * ay) / CS2 + W9[i] * psi * divu;
}

/* Sec. 3.2: flow equilibrium and forcing. */
static double h_eq(int i, double p, double rho, double ux, double uy)
{
    double pre = (i == 0) ? p / CS2 * (W9[0] - 1.0) : p / CS2 * W9[i];
    return pre + rho * s_i(i, ux, uy);
}

static double h_src(int i, double S, double Fx, double Fy, double rfx, double rfy,
                    double ux, double uy, double Ftx, double Fty)
{
    double cu = CX[i] * ux + CY[i] * uy;
    double cF = CX[i] * Ftx + CY[i] * Fty;
    double uF = ux * Ftx + uy * Fty;
    /* (u Ft + Ft u):(c c - cs2 I) / (2 cs2^2) = [(c.u)(c.Ft) - cs2 u.Ft] / cs2^2 (R12) */
    return W9[i] * (S + (CX[i] * (Fx + rfx) + CY[i] * (Fy + rfy)) / CS2 +
                    (cu * cF - CS2 * uF) / (CS2 * CS2));
}

/* Sec. 3.3: enthalpy equilibrium. */
static double g_eq(int i, double H, double T, double cp, double Cref, double ux, double uy)
{
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    if (i == 0)
        return H - Cref * T + W9[0] * cp * T * (Cref / cp - uu / (2.0 * CS2));
    return W9[i] * cp * T * (Cref / cp + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
}

/* Sec. 3.4: potential equilibrium (D2Q5). */
static double l_eq(int i, double phi)
{
    return (i == 0) ? (W5[0] - 1.0) * phi : W5[i] * phi;
}

/* Exported for the moment-identity tests (all four equilibria and both
 * forcing terms at one point; q-arrays are caller-owned). */
void orc_pointwise(double psi, double ux, double uy, double p, double rho, double H,
                   double T, double cp, double Cref, double phi, double S, double Fx,
                   double Fy, double rfx, double rfy, double Ftx, double Fty,
                   double dtx, double dty, double lam, double nxv, double nyv,
                   double divu, double *feq, double *fsrc, double *heq, double *hsrc,
                   double *geq, double *leq)
{
    build_lattice();
    for (int i = 0; i < 9; i++) {
        feq[i] = f_eq(i, psi, ux, uy);
        fsrc[i] = f_src(i, psi, dtx, dty, lam, nxv, nyv, divu);
        heq[i] = h_eq(i, p, rho, ux, uy);
        hsrc[i] = h_src(i, S, Fx, Fy, rfx, rfy, ux, uy, Ftx, Fty);
        geq[i] = g_eq(i, H, T, cp, Cref, ux, uy);
    }
    for (int i = 0; i < 5; i++) leq[i] = l_eq(i, phi);
}

/* ------------------------------------------------------------------ */
/* Finite-difference stencils (Eqs. eqtidi1, eqtidi2) with the wall     */
/* ghost rules (R17, R19).                                              */
/* ------------------------------------------------------------------ */
enum { GH_COPY = 0, GH_PSI = 1, GH_PHI = 2 };

static double at(const orc_state *s, const double *z, int kind, int x, int y)
{
    int nx = s->nx, ny = s->ny;
    int xx = (x < 0) ? x + nx : (x >= nx ? x - nx : x);    /* periodic in x */
    if (y >= 0 && y < ny) return z[(long)y * nx + xx];
    int yi = (y < 0) ? 0 : ny - 1;
    double zi = z[(long)yi * nx + xx];
    if (kind == GH_PSI)
        return (y < 0) ? zi + s->D.wet * zi * (1.0 - zi) : zi;
    if (kind == GH_PHI)
        return 2.0 * ((y < 0) ? s->D.phi_bot : s->D.phi_top) - zi;
    return zi;
}

static void grad(const orc_state *s, const double *z, int kind, int x, int y,
                 double *gx, double *gy)
{
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < 9; i++) {
        double v = at(s, z, kind, x + CX[i], y + CY[i]);
        sx += W9[i] * CX[i] * v;
        sy += W9[i] * CY[i] * v;
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
}

static double lap(const orc_state *s, const double *z, int kind, int x, int y)
{
    double z0 = at(s, z, kind, x, y);
    double acc = 0.0;
    for (int i = 1; i < 9; i++)
        acc += 2.0 * W9[i] * (at(s, z, kind, x + CX[i], y + CY[i]) - z0);
    return acc / CS2;
}

/* Exported for the stencil tests: gradient and Laplacian of an arbitrary
 * field on an nx x ny lattice, ghost kind 0 (copy), 1 (wetting), 2 (phi). */
void orc_stencils(int32_t nx, int32_t ny, const double *z, int32_t kind, double wet,
                  double phi_bot, double phi_top, double *gx, double *gy, double *lp)
{
    build_lattice();
    orc_state s;
    memset(&s, 0, sizeof s);
    s.nx = nx; s.ny = ny; s.N = (long)nx * ny;
    s.D.wet = wet; s.D.phi_bot = phi_bot; s.D.phi_top = phi_top;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long k = (long)y * nx + x;
            grad(&s, z, kind, x, y, &gx[k], &gy[k]);
            lp[k] = lap(&s, z, kind, x, y);
        }
}

/* ------------------------------------------------------------------ */
/* State management.                                                    */
/* ------------------------------------------------------------------ */
static double *zeros(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

orc_state *orc_create(const orc_params *P)
{
    build_lattice();
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->P = *P;
    if (orc_derive(P, &s->D) != 0) { free(s); return NULL; }
    s->nx = P->nx; s->ny = P->ny; s->N = (long)P->nx * P->ny;
    s->f = zeros(9 * s->N); s->h = zeros(9 * s->N); s->g = zeros(9 * s->N);
    s->l = zeros(5 * s->N);
    s->fs_prev = zeros(s->N); s->mdot_prev = zeros(s->N); s->Q_prev = zeros(s->N);
    s->psiux_prev = zeros(s->N); s->psiuy_prev = zeros(s->N);
    s->p_prev = zeros(s->N); s->S_prev = zeros(s->N); s->sigma_n = zeros(s->N);
    s->t_fre = -1;
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    free(s->f); free(s->h); free(s->g); free(s->l);
    free(s->fs_prev); free(s->mdot_prev); free(s->Q_prev);
    free(s->psiux_prev); free(s->psiuy_prev); free(s->p_prev); free(s->S_prev);
    free(s->sigma_n);
    free(s);
}

void orc_get_derived(const orc_state *s, orc_derived *D) { *D = s->D; }
int64_t orc_get_step(const orc_state *s) { return s->step; }

/* ------------------------------------------------------------------ */
/* Local macroscopic quantities at time n (a1).                         */
/* ------------------------------------------------------------------ */
typedef struct {
    double psi, H, fl, T, fs, rho, mu, kth, eps, sig, cp, phi;
} macro;

static void cell_macros(const orc_state *s, long k, macro *m)
{
    const long N = s->N;
    double sf = 0.0;
    for (int i = 0; i < 9; i++) sf += s->f[i * N + k];
    /* Eq. (Computed_psi): psi = sum f + psi div(u)/2, div u = lagged mdot (R7, R8) */
    m->psi = sf / (1.0 - 0.5 * s->mdot_prev[k]);
    double sg = 0.0;
    for (int i = 0; i < 9; i++) sg += s->g[i * N + k];
    /* Sec. 3.3: H = sum g + rho C_p T mdot / 2 with the lagged product (R7) */
    m->H = sg + 0.5 * s->Q_prev[k];
    double cp_lev = chi(s->fs_prev[k], m->psi, s->D.cp);
    orc_enthalpy_inversion(m->H, m->psi, cp_lev, s->P.T_m, s->D.L, &m->fl, &m->T);
    m->fs = m->psi * (1.0 - m->fl);                       /* R6 */
    m->rho = chi(m->fs, m->psi, s->D.rho);
    m->mu = chi(m->fs, m->psi, s->D.mu);
    m->kth = chi(m->fs, m->psi, s->D.kth);
    m->eps = chi(m->fs, m->psi, s->D.eps);
    m->sig = chi(m->fs, m->psi, s->D.sig);
    m->cp = chi(m->fs, m->psi, s->D.cp);
    double sl = 0.0;
    for (int i = 1; i < 5; i++) sl += s->l[i * N + k];
    m->phi = sl / (1.0 - W5[0]);                          /* Eq. (Computed_phi) */
}

/* ------------------------------------------------------------------ */
/* Streaming with wall treatments (Algorithm 1; R18).                   */
/* post: post-collision populations; out: populations at time n+1.      */
/* wall_bot/wall_top: 0 bounce-back, 1 anti-bounce-back with value.     */
/* ------------------------------------------------------------------ */
static void stream9(const orc_state *s, const double *post, double *out,
                    int bot_anti, double bot_val, int top_anti, double top_val)
{
    const int nx = s->nx, ny = s->ny;
    const long N = s->N;
    for (int i = 0; i < 9; i++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long k = (long)y * nx + x;
                int xs = ((x - CX[i]) % nx + nx) % nx;
                int ys = y - CY[i];
                double v;
                if (ys >= 0 && ys < ny) {
                    v = post[i * N + (long)ys * nx + xs];
                } else {
                    int o = OPP[i];
                    double back = post[o * N + k];
                    int anti = (ys < 0) ? bot_anti : top_anti;
                    double val = (ys < 0) ? bot_val : top_val;
                    v = anti ? -back + 2.0 * W9[o] * val : back;
                }
                out[i * N + k] = v;
            }
}

static void stream5(const orc_state *s, const double *post, double *out)
{
    const int nx = s->nx, ny = s->ny;
    const long N = s->N;
    for (int i = 0; i < 5; i++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long k = (long)y * nx + x;
                int xs = ((x - CX5[i]) % nx + nx) % nx;
                int ys = y - CY5[i];
                double v;
                if (ys >= 0 && ys < ny) {
                    v = post[i * N + (long)ys * nx + xs];
                } else {
                    int o = OPP5[i];
                    double phiw = (ys < 0) ? s->D.phi_bot : s->D.phi_top;
                    v = -post[o * N + k] + 2.0 * W5[o] * phiw;   /* electrodes */
                }
                out[i * N + k] = v;
            }
}

/* One extra sweep of the potential LB with sigma frozen at time n (R15). */
static void potential_sweep(orc_state *s)
{
    const long N = s->N;
    double *post = zeros(5 * N);
    for (long k = 0; k < N; k++) {
        double sl = 0.0;
        for (int i = 1; i < 5; i++) sl += s->l[i * N + k];
        double phi = sl / (1.0 - W5[0]);
        double tau_l = s->sigma_n[k] / CS2 + 0.5;
        for (int i = 0; i < 5; i++) {
            double li = s->l[i * N + k];
            post[i * N + k] = li - (li - l_eq(i, phi)) / tau_l;
        }
    }
    stream5(s, post, s->l);
    free(post);
}

/* ------------------------------------------------------------------ */
/* One time step n -> n+1 (Algorithm 1 under reading R1).               */
/* ------------------------------------------------------------------ */
static void one_step(orc_state *s)
{
    const int nx = s->nx, ny = s->ny;
    const long N = s->N;
    const orc_derived *D = &s->D;

    double *psi = zeros(N), *H = zeros(N), *fs = zeros(N), *T = zeros(N);
    double *rho = zeros(N), *mu = zeros(N), *kth = zeros(N), *eps = zeros(N);
    double *sig = zeros(N), *cp = zeros(N), *phi = zeros(N), *mdot = zeros(N);
    double *fpost = zeros(9 * N), *hpost = zeros(9 * N), *gpost = zeros(9 * N);
    double *lpost = zeros(5 * N);
    double *psiux = zeros(N), *psiuy = zeros(N), *pn = zeros(N), *Sn = zeros(N), *Qn = zeros(N);

    /* a1: macroscopic fields at time n */
    for (long k = 0; k < N; k++) {
        macro m;
        cell_macros(s, k, &m);
        psi[k] = m.psi; H[k] = m.H; fs[k] = m.fs; T[k] = m.T;
        rho[k] = m.rho; mu[k] = m.mu; kth[k] = m.kth; eps[k] = m.eps;
        sig[k] = m.sig; cp[k] = m.cp; phi[k] = m.phi;
        /* Eq. (ns1) with an explicit Euler derivative of f_s */
        mdot[k] = (1.0 - D->rho[0] / D->rho[1]) * (fs[k] - s->fs_prev[k]);
    }

    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long k = (long)y * nx + x;
            /* a2: stencils */
            double gpsix, gpsiy, grhox, grhoy, gepsx, gepsy, gphix, gphiy;
            double gpx, gpy, gSx, gSy;
            grad(s, psi, GH_PSI, x, y, &gpsix, &gpsiy);
            double lpsi = lap(s, psi, GH_PSI, x, y);
            grad(s, rho, GH_COPY, x, y, &grhox, &grhoy);
            grad(s, eps, GH_COPY, x, y, &gepsx, &gepsy);
            grad(s, phi, GH_PHI, x, y, &gphix, &gphiy);
            double lphi = lap(s, phi, GH_PHI, x, y);
            grad(s, s->p_prev, GH_COPY, x, y, &gpx, &gpy);
            grad(s, s->S_prev, GH_COPY, x, y, &gSx, &gSy);

            /* a3: forces.  Chemical potential with psi_l = 1, psi_g = 0. */
            double ps = psi[k];
            double muc = 4.0 * D->beta * (ps - 1.0) * (ps - 0.0) * (ps - 0.5) - D->kappa * lpsi;
            double Fsx = muc * gpsix, Fsy = muc * gpsiy;                     /* Eq. (Fs) */
            double Ex = -gphix, Ey = -gphiy;                                  /* E = -grad phi */
            double qv = -(gepsx * gphix + gepsy * gphiy + eps[k] * lphi);     /* div(eps E) */
            double E2 = Ex * Ex + Ey * Ey;
            double Fex = qv * Ex - 0.5 * E2 * gepsx;                          /* Eq. (Fe) */
            double Fey = qv * Ey - 0.5 * E2 * gepsy;
            double Fx = Fsx + Fex, Fy = Fsy + Fey;                            /* F_b = 0 */

            /* a4: flow macros (Sec. 3.2) */
            double jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; i++) {
                jx += CX[i] * s->h[i * N + k];
                jy += CY[i] * s->h[i * N + k];
            }
            double r = rho[k];
            double usx = (jx + 0.5 * Fx) / r, usy = (jy + 0.5 * Fy) / r;     /* rho u* */
            double fx = fs[k] * (0.0 - usx), fy = fs[k] * (0.0 - usy);      /* R11 */
            double ux = usx + 0.5 * fx, uy = usy + 0.5 * fy;                  /* Eq. (Computed_u) */
            double rfx = r * fx, rfy = r * fy;
            double S = r * mdot[k] + (ux * grhox + uy * grhoy);
            double Ftx = Fx - gpx + CS2 * grhox + CS2 * gSx;                  /* R9 */
            double Fty = Fy - gpy + CS2 * grhoy + CS2 * gSy;
            double uF = ux * Ftx + uy * Fty;
            double R0 = W9[0] * (S - uF / CS2);                               /* R10 */
            double tau_h = mu[k] / r / CS2 + 0.5;
            double sh = 0.0;
            for (int i = 1; i < 9; i++) sh += s->h[i * N + k];
            double p = CS2 / (1.0 - W9[0]) * (sh + 0.5 * S + tau_h * R0 + r * s_i(0, ux, uy));

            /* a7: flow collision */
            for (int i = 0; i < 9; i++) {
                double hi = s->h[i * N + k];
                double Ri = h_src(i, S, Fx, Fy, rfx, rfy, ux, uy, Ftx, Fty);
                hpost[i * N + k] = hi - (hi - h_eq(i, p, r, ux, uy)) / tau_h +
                                   (1.0 - 1.0 / (2.0 * tau_h)) * Ri;
            }

            /* a5: phase-field collision (Sec. 3.1) */
            double pux = ps * ux, puy = ps * uy;
            double dtx = pux - s->psiux_prev[k], dty = puy - s->psiuy_prev[k];
            double gn = sqrt(gpsix * gpsix + gpsiy * gpsiy);
            double nxv = gpsix / (gn + 1e-4), nyv = gpsiy / (gn + 1e-4);    /* R2 */
            double lam = 4.0 * ps * (1.0 - ps) / s->P.W;
            for (int i = 0; i < 9; i++) {
                double fi = s->f[i * N + k];
                double Fi = f_src(i, ps, dtx, dty, lam, nxv, nyv, mdot[k]);
                fpost[i * N + k] = fi - (fi - f_eq(i, ps, ux, uy)) / D->tau_f +
                                   (1.0 - 1.0 / (2.0 * D->tau_f)) * Fi;
            }

            /* a8: enthalpy collision (Sec. 3.3, R13) */
            double tau_g = kth[k] / (r * D->Cref * CS2) + 0.5;
            double Q = r * cp[k] * T[k] * mdot[k];
            for (int i = 0; i < 9; i++) {
                double gi = s->g[i * N + k];
                gpost[i * N + k] = gi - (gi - g_eq(i, H[k], T[k], cp[k], D->Cref, ux, uy)) / tau_g +
                                   (1.0 - 1.0 / (2.0 * tau_g)) * (W9[i] * Q);
            }

            /* a6: potential collision (Sec. 3.4) */
            double tau_l = sig[k] / CS2 + 0.5;
            for (int i = 0; i < 5; i++) {
                double li = s->l[i * N + k];
                lpost[i * N + k] = li - (li - l_eq(i, phi[k])) / tau_l;
            }

            psiux[k] = pux; psiuy[k] = puy; pn[k] = p; Sn[k] = S; Qn[k] = Q;
        }

    /* a9: streaming and walls (Algorithm 1: BB for f, h; anti-BB for g
     * at the cold wall, BB at the top; anti-BB for l at both electrodes) */
    stream9(s, fpost, s->f, 0, 0.0, 0, 0.0);
    stream9(s, hpost, s->h, 0, 0.0, 0, 0.0);
    stream9(s, gpost, s->g, 1, D->Cref * s->P.T_w, 0, 0.0);
    stream5(s, lpost, s->l);

    memcpy(s->fs_prev, fs, N * sizeof(double));
    memcpy(s->mdot_prev, mdot, N * sizeof(double));
    memcpy(s->Q_prev, Qn, N * sizeof(double));
    memcpy(s->psiux_prev, psiux, N * sizeof(double));
    memcpy(s->psiuy_prev, psiuy, N * sizeof(double));
    memcpy(s->p_prev, pn, N * sizeof(double));
    memcpy(s->S_prev, Sn, N * sizeof(double));
    memcpy(s->sigma_n, sig, N * sizeof(double));

    for (int j = 1; j < s->P.k_e; j++) potential_sweep(s);
    s->step += 1;

    free(psi); free(H); free(fs); free(T); free(rho); free(mu); free(kth); free(eps);
    free(sig); free(cp); free(phi); free(mdot); free(fpost); free(hpost); free(gpost);
    free(lpost); free(psiux); free(psiuy); free(pn); free(Sn); free(Qn);
}

void orc_step(orc_state *s, int64_t n)
{
    for (int64_t j = 0; j < n; j++) one_step(s);
}

/* ------------------------------------------------------------------ */
/* Initial state (Sec. 2 and Algorithm 1's initialisation).             */
/* The droplet is at rest and at T_init, every population is at its     */
/* equilibrium, the potential is linear between the electrodes, and    */
/* `presolve` potential sweeps relax it around the droplet first.       */
/* ------------------------------------------------------------------ */
int orc_init_psi(orc_state *s, const double *psi0, int32_t presolve)
{
    const int nx = s->nx, ny = s->ny;
    const long N = s->N;
    const orc_derived *D = &s->D;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long k = (long)y * nx + x;
            double ps = psi0[k];
            double cpm = chi(0.0, ps, D->cp);
            double T0 = s->P.T_init;
            double H0 = cpm * T0 + ps * D->L;          /* all latent heat still held */
            double phi0 = D->phi_bot + (D->phi_top - D->phi_bot) * (y + 0.5) / ny;
            for (int i = 0; i < 9; i++) {
                s->f[i * N + k] = f_eq(i, ps, 0.0, 0.0);
                s->h[i * N + k] = h_eq(i, 0.0, chi(0.0, ps, D->rho), 0.0, 0.0);
                s->g[i * N + k] = g_eq(i, H0, T0, cpm, D->Cref, 0.0, 0.0);
            }
            for (int i = 0; i < 5; i++) s->l[i * N + k] = l_eq(i, phi0);
            s->fs_prev[k] = 0.0; s->mdot_prev[k] = 0.0; s->Q_prev[k] = 0.0;
            s->psiux_prev[k] = 0.0; s->psiuy_prev[k] = 0.0;
            s->p_prev[k] = 0.0; s->S_prev[k] = 0.0;
            s->sigma_n[k] = chi(0.0, ps, D->sig);
        }
    for (int j = 0; j < presolve; j++) potential_sweep(s);
    s->step = 0;
    s->t_fre = -1;
    return 0;
}

/* Circular droplet of radius R centred at (xc, yc): psi = 1/2 + 1/2 tanh(2(R-r)/W). */
int orc_init_droplet(orc_state *s, double R, double xc, double yc, int32_t presolve)
{
    const int nx = s->nx, ny = s->ny;
    double *psi0 = zeros(s->N);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double dx = x - xc, dy = y - yc;
            double r = sqrt(dx * dx + dy * dy);
            psi0[(long)y * nx + x] = 0.5 + 0.5 * tanh(2.0 * (R - r) / s->P.W);
        }
    int rc = orc_init_psi(s, psi0, presolve);
    free(psi0);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Field access (tests).  Field ids follow the library's numbering.      */
/* ------------------------------------------------------------------ */
enum {
    F_POP_F = 0, F_POP_H = 1, F_POP_G = 2, F_POP_L = 3, F_FS_PREV = 4, F_MDOT_PREV = 5,
    F_Q_PREV = 6, F_PSIUX = 7, F_PSIUY = 8, F_P = 9, F_S = 10, F_PSI = 11, F_FSOLID = 12,
    F_T = 13, F_PHI = 14, F_HTOT = 15, F_SIGMA = 16
};

static double *field_ptr(orc_state *s, int id, int *planes)
{
    *planes = 1;
    switch (id) {
    case F_POP_F: *planes = 9; return s->f;
    case F_POP_H: *planes = 9; return s->h;
    case F_POP_G: *planes = 9; return s->g;
    case F_POP_L: *planes = 5; return s->l;
    case F_FS_PREV: return s->fs_prev;
    case F_MDOT_PREV: return s->mdot_prev;
    case F_Q_PREV: return s->Q_prev;
    case F_PSIUX: return s->psiux_prev;
    case F_PSIUY: return s->psiuy_prev;
    case F_P: return s->p_prev;
    case F_S: return s->S_prev;
    case F_SIGMA: return s->sigma_n;
    default: return NULL;
    }
}

int orc_get_field(orc_state *s, int32_t id, double *out)
{
    int planes;
    double *src = field_ptr(s, id, &planes);
    if (src) {
        memcpy(out, src, (size_t)planes * s->N * sizeof(double));
        return 0;
    }
    if (id < F_PSI || id > F_HTOT) return -1;
    for (long k = 0; k < s->N; k++) {
        macro m;
        cell_macros(s, k, &m);
        out[k] = (id == F_PSI) ? m.psi : (id == F_FSOLID) ? m.fs : (id == F_T) ? m.T
               : (id == F_PHI) ? m.phi : m.H;
    }
    return 0;
}

int orc_set_field(orc_state *s, int32_t id, const double *in)
{
    int planes;
    double *dst = field_ptr(s, id, &planes);
    if (!dst) return -1;
    memcpy(dst, in, (size_t)planes * s->N * sizeof(double));
    return 0;
}

/* ------------------------------------------------------------------ */
/* Observables (a10).  Definitions (the paper gives none numerically):  */
/*   mass = sum psi, enthalpy = sum H, solid = sum f_s, charge = sum q_v */
/*   frozen_fraction = solid / mass                                      */
/*   height: highest psi = 1/2 crossing of any column, from y = -1/2     */
/*   width: widest psi = 1/2 extent of any row; R_tr = half of row 0's   */
/*   front: lowest f_s = 1/2 crossing above a frozen bottom cell on     */
/*          column nx/2 (the front rising from the cold wall)           */
/*   t_fre: first observed step with frozen_fraction >= 0.99             */
/* ------------------------------------------------------------------ */
static double col_crossing(const double *z, int nx, int ny, int x)
{
    /* highest y with z(y) >= 1/2 > z(y+1), linearly interpolated */
    if (z[(long)(ny - 1) * nx + x] >= 0.5) return (double)ny;
    double best = 0.0;
    for (int y = 0; y + 1 < ny; y++) {
        double a = z[(long)y * nx + x], b = z[(long)(y + 1) * nx + x];
        if (a >= 0.5 && b < 0.5) {
            double hgt = y + (a - 0.5) / (a - b) + 0.5;
            if (hgt > best) best = hgt;
        }
    }
    return best;
}

static double front_crossing(const double *z, int nx, int ny, int x)
{
    /* freezing front rising from the cold wall: lowest y with
     * z(y) >= 1/2 > z(y+1) on a column whose bottom cell is frozen */
    if (z[x] < 0.5) return 0.0;
    for (int y = 0; y + 1 < ny; y++) {
        double a = z[(long)y * nx + x], b = z[(long)(y + 1) * nx + x];
        if (a >= 0.5 && b < 0.5) return y + (a - 0.5) / (a - b) + 0.5;
    }
    return (double)ny;
}

static double row_extent(const double *psi, int nx, int y)
{
    const double *r = psi + (long)y * nx;
    int any = 0;
    double left = 1e300, right = -1e300;
    for (int x = 0; x < nx; x++) {
        if (r[x] >= 0.5) any = 1;
        if (x >= 1 && r[x] >= 0.5 && r[x - 1] < 0.5) {
            double xl = (x - 1) + (0.5 - r[x - 1]) / (r[x] - r[x - 1]);
            if (xl < left) left = xl;
        }
        if (x + 1 < nx && r[x] >= 0.5 && r[x + 1] < 0.5) {
            double xr = x + (r[x] - 0.5) / (r[x] - r[x + 1]);
            if (xr > right) right = xr;
        }
    }
    if (!any) return 0.0;
    if (left > 1e299 || right < -1e299) return (double)nx;
    return right - left;
}

/* R24: local substrate heat flux Qdot(x) = -k dT/dy at the substrate
 * (Sec. 4.3), one value per column.  Needs ny >= 3. */
int orc_heat_flux(const orc_state *s, double *out)
{
    if (s->ny < 3) return -1;
    for (int x = 0; x < s->nx; x++) {
        macro m0, m1, m2;
        cell_macros(s, x, &m0);
        cell_macros(s, (long)s->nx + x, &m1);
        cell_macros(s, 2L * s->nx + x, &m2);
        out[x] = -m0.kth * (4.0 * m1.T - m2.T - 3.0 * m0.T) / 2.0;
    }
    return 0;
}

int orc_observables(orc_state *s, orc_obs *o)
{
    const int nx = s->nx, ny = s->ny;
    const long N = s->N;
    double *psi = zeros(N), *fsv = zeros(N), *eps = zeros(N), *phi = zeros(N), *Hv = zeros(N);
    int bad = 0;
    for (long k = 0; k < N; k++) {
        macro m;
        cell_macros(s, k, &m);
        psi[k] = m.psi; fsv[k] = m.fs; eps[k] = m.eps; phi[k] = m.phi; Hv[k] = m.H;
        if (!isfinite(m.psi) || !isfinite(m.H)) bad = 1;
    }
    /* R25: liquid-weighted mean speed from the stored psi u */
    double liq = 0.0, liq_u = 0.0;
    for (long k = 0; k < N; k++) {
        double w = psi[k] - fsv[k];
        if (w > 0.0) {
            double sp = sqrt(s->psiux_prev[k] * s->psiux_prev[k] + s->psiuy_prev[k] * s->psiuy_prev[k]);
            liq += w;
            liq_u += w * sp / psi[k];
        }
    }
    /* R24: substrate heat flux summed over x */
    double qsum = 0.0;
    if (ny >= 3) {
        double *q = zeros(nx);
        orc_heat_flux(s, q);
        for (int x = 0; x < nx; x++) qsum += q[x];
        free(q);
    }
    double mass = 0.0, enth = 0.0, solid = 0.0, charge = 0.0;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long k = (long)y * nx + x;
            double gex, gey, gphx, gphy;
            grad(s, eps, GH_COPY, x, y, &gex, &gey);
            grad(s, phi, GH_PHI, x, y, &gphx, &gphy);
            double lphi = lap(s, phi, GH_PHI, x, y);
            double qv = -(gex * gphx + gey * gphy + eps[k] * lphi);
            mass += psi[k]; enth += Hv[k]; solid += fsv[k]; charge += qv;
        }
    double height = 0.0, width = 0.0;
    for (int x = 0; x < nx; x++) {
        double hgt = col_crossing(psi, nx, ny, x);
        if (hgt > height) height = hgt;
    }
    for (int y = 0; y < ny; y++) {
        double w = row_extent(psi, nx, y);
        if (w > width) width = w;
    }
    o->step = s->step;
    o->Fo = s->P.alpha_l * (double)s->step / (s->P.R0 * s->P.R0);
    o->mass = mass; o->enthalpy = enth; o->charge = charge; o->solid = solid;
    o->frozen_fraction = (mass != 0.0) ? solid / mass : 0.0;
    o->height = height;
    o->width = width;
    o->aspect = (width > 0.0) ? height / width : 0.0;
    o->R_tr = 0.5 * row_extent(psi, nx, 0);
    o->front = front_crossing(fsv, nx, ny, nx / 2);
    if (s->t_fre < 0 && o->frozen_fraction >= 0.99) s->t_fre = s->step;
    o->t_fre = s->t_fre;
    o->Fo_fre = (s->t_fre >= 0) ? s->P.alpha_l * (double)s->t_fre / (s->P.R0 * s->P.R0) : -1.0;
    o->status = bad ? -3 : 0;
    o->reserved = 0;
    o->Pe = (liq > 0.0) ? 2.0 * s->P.R0 * (liq_u / liq) / s->P.alpha_l : 0.0;
    o->Qdot = qsum;
    free(psi); free(fsv); free(eps); free(phi); free(Hv);
    return o->status;
}
