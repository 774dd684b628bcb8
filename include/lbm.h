/*
 * lbm.h -- C ABI of the GB300 phase-field lattice Boltzmann library for the
 * freezing of a wetting droplet under a uniform electric field
 * (Huang, Li, Che, Chai, Wang, Shi, arXiv 2410.06657).
 *
 * One time step advances four coupled lattice Boltzmann systems on an
 * nx x ny lattice (Sec. 3, Algorithm 1):
 *   f  D2Q9 Allen-Cahn phase field psi            (Sec. 3.1, Eq. LB-PF)
 *   h  D2Q9 incompressible flow with a mass source (Sec. 3.2, Eq. LB_flow)
 *   g  D2Q9 total enthalpy H -> T, solid fraction  (Sec. 3.3, Eqs. LB_H, Hfl)
 *   l  D2Q5 electric potential phi                 (Sec. 3.4, Eq. LB_phi)
 * with the isotropic gradient/Laplacian stencils (Eqs. eqtidi1-2), the
 * surface-tension and leaky-dielectric forces (Eqs. Fs, Fe), and the wall
 * treatments of Algorithm 1.  x is periodic; walls sit at y = -1/2 (cold
 * substrate at T_w, bottom electrode phi = 0, wetting at angle theta) and at
 * y = ny - 1/2 (adiabatic, top electrode phi = E0 * ny, neutral wetting).
 *
 * Conventions for every call:
 *   - Returns LBM_OK (0) or a negative LBM_ERR_* code (lbm_presolve may
 *     also return the positive warning LBM_WARN_NOT_CONVERGED); nothing
 *     throws.
 *   - The library owns all device memory of a handle; callers own every
 *     host buffer they pass.  It is only read or written during the call,
 *     except by the asynchronous transfers of lbm_import_state,
 *     lbm_observables_to_host and lbm_observables_deferred, which use it
 *     until the handle's stream has passed them (lbm_sync).
 *   - A handle is bound to one CUDA stream and to the device that was
 *     current at lbm_create (make it current for every call on the handle),
 *     and is not thread-safe.  Calls that only enqueue work (lbm_step)
 *     return before the GPU finishes; calls that return data to the host
 *     synchronise that stream.
 *   - All arithmetic runs in the library's CUDA kernels; there is no CPU
 *     path.  A call made without a usable GPU returns LBM_ERR_CUDA.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage / arithmetic precision of a handle. */
enum {
    LBM_FP64 = 0,  /* populations and arithmetic in double                      */
    LBM_FP32 = 1,  /* populations and arithmetic in float                       */
    LBM_FP16S = 2  /* h, g, l stored as half after subtracting a reference      */
                   /* state (weight-shifted); g and l rounded stochastically,   */
                   /* h to nearest; the phase-field populations f stay in       */
                   /* float; arithmetic in float                                */
};

/* Return codes. */
enum {
    LBM_OK = 0,
    LBM_ERR_BADPARAM = -1,   /* a parameter is out of range (see lbm_params)   */
    LBM_ERR_OOM = -2,        /* device allocation failed                       */
    LBM_ERR_DIVERGED = -3,   /* a non-finite psi or H was seen; the handle     */
                             /* refuses further steps                          */
    LBM_ERR_CUDA = -4,       /* a CUDA call failed (message: lbm_last_error)   */
    LBM_ERR_STATE = -5,      /* call out of order (e.g. step before init)      */
    LBM_WARN_NOT_CONVERGED = 1  /* warning, lbm_presolve only: the tolerance  */
                                /* was not met within max_sweeps              */
};

/*
 * Problem parameters: the paper's dimensionless numbers plus the lattice
 * choices it leaves open.  All quantities are in lattice units
 * (dx = dt = 1, Sec. 3.1).  Derived quantities (Sec. 2 and Sec. 4):
 *   rho_g = rho_l / rho_lg, rho_s = rho_l * rho_sl, mu_g = mu_l / mu_lg,
 *   mu_s = mu_l; L = cp_l (T_m - T_w) / Ste; k_phase = rho C_p alpha with
 *   alpha_g = alpha_l / alpha_lg and alpha_s = alpha_l * alpha_sl;
 *   eps_l = eps_s = S_eps * eps_g; sigma_l = sigma_s = R_sigma * sigma_g;
 *   E0 = sqrt(CaE * gamma / (eps_g * R0)) (CaE = eps_e E0^2 R / gamma, Sec. 4);
 *   kappa = 3 gamma W / 2, beta = 12 gamma / W (Sec. 2);
 *   C_p,ref = 2 cp_s cp_l / (cp_s + cp_l) (Sec. 3.3).
 * Validity (else LBM_ERR_BADPARAM): nx, ny > 0 with 32 x (nx rounded up to a
 * multiple of 32) x ny < 2^32 (about 134 million cells); k_e >= 1; precision one of
 * LBM_FP*; W, M, rho_l, rho_lg, rho_sl, mu_l, mu_lg, Ste, alpha_l, alpha_lg,
 * alpha_sl, cp_*, R_sigma, S_eps, eps_g, sigma_g, R0 > 0; gamma, CaE >= 0;
 * 0 < theta_deg < 180; T_m >= T_w.  These keep every relaxation time above
 * 1/2 in every phase and every mixture.
 */
typedef struct lbm_params {
    int32_t nx, ny;      /* lattice size                                     */
    int32_t k_e;         /* potential sweeps per time step (>= 1)            */
    int32_t precision;   /* LBM_FP64 | LBM_FP32 | LBM_FP16S                  */
    double W;            /* interface width                                  */
    double M;            /* phase-field mobility (tau_f = M / c_s^2 + 1/2)   */
    double gamma;        /* liquid-gas surface tension                       */
    double rho_l;        /* liquid density                                   */
    double rho_lg;       /* rho_l / rho_g                                    */
    double rho_sl;       /* rho_s / rho_l                                    */
    double mu_l;         /* liquid dynamic viscosity                         */
    double mu_lg;        /* mu_l / mu_g (the paper's viscosity ratio)        */
    double Ste;          /* Stefan number cp_l (T_m - T_w) / L               */
    double alpha_l;      /* liquid thermal diffusivity                       */
    double alpha_lg;     /* alpha_l / alpha_g                                */
    double cp_l, cp_s, cp_g;   /* specific heats                             */
    double T_m;          /* melting temperature                              */
    double T_w;          /* cold-wall temperature                            */
    double T_init;       /* initial temperature of the whole domain          */
    double CaE;          /* electric capillary number                        */
    double R_sigma;      /* conductivity ratio R = sigma_l / sigma_g         */
    double S_eps;        /* permittivity ratio S = eps_l / eps_g             */
    double eps_g;        /* gas permittivity                                 */
    double sigma_g;      /* gas conductivity (tau_l = sigma / c_s^2 + 1/2)   */
    double R0;           /* reference radius in CaE and Fo = alpha_l t / R0^2 */
    double theta_deg;    /* static contact angle on the bottom wall          */
    double alpha_sl;     /* alpha_s / alpha_l (1: the solid conducts like the */
                         /* liquid; Table 1 property sets differ)            */
} lbm_params;

/*
 * Observables of one instance.  The paper measures these from
 * its fields but gives no discrete definition; the library's are:
 *   mass = sum psi, enthalpy = sum H, solid = sum f_s, charge = sum q_v with
 *   q_v = div(eps E) by the product rule.  The per-cell terms are evaluated
 *   in the handle's arithmetic precision; the 32 cells of one tile row are
 *   summed in that precision (FP32 for LBM_FP32 and LBM_FP16S), and every
 *   level above -- rows, tiles, groups of tiles, the lattice -- in FP64;
 *   frozen_fraction = solid / mass;
 *   height = highest interpolated psi = 1/2 crossing of any column,
 *            measured from the wall at y = -1/2;
 *   width  = widest interpolated psi = 1/2 extent of any row;
 *   aspect = height / width; R_tr = half of row 0's extent (contact line);
 *   front  = lowest interpolated f_s = 1/2 crossing on column nx/2 above a
 *            frozen bottom cell (0 if that cell is not frozen);
 *   t_fre  = first step at which an observables call saw
 *            frozen_fraction >= 0.99 (-1 until then), Fo_fre its Fourier number;
 *   status = LBM_OK or LBM_ERR_DIVERGED (non-finite psi or H anywhere);
 *   Pe     = 2 R0 u_d / alpha_l (Sec. 4.3, Peclet number with D_d = 2 R0),
 *            u_d = mean of |psi u| / psi weighted by the liquid content
 *            psi - f_s, from the psi u stored by the last step (0 without
 *            liquid);
 *   Qdot   = sum over x of the substrate heat flux of
 *            lbm_substrate_heat_flux (0 when ny < 3).
 */
typedef struct lbm_obs {
    int64_t step;
    double Fo;
    double mass, enthalpy, charge, solid, frozen_fraction;
    double height, width, aspect, R_tr, front;
    int64_t t_fre;
    double Fo_fre;
    int32_t status;
    int32_t reserved;
    double Pe;
    double Qdot;
} lbm_obs;

/* Field ids for lbm_get_field / lbm_set_field.  Arrays are host doubles,
 * row-major [plane][y][x] with x fastest, planes as stated. */
enum {
    LBM_FIELD_F = 0,        /* 9 planes: phase-field populations f_i at time n   */
    LBM_FIELD_H = 1,        /* 9 planes: flow populations h_i                    */
    LBM_FIELD_G = 2,        /* 9 planes: enthalpy populations g_i                */
    LBM_FIELD_L = 3,        /* 5 planes: potential populations l_i               */
    LBM_FIELD_FS_PREV = 4,  /* solid fraction of the previous step               */
    LBM_FIELD_MDOT_PREV = 5,/* mass source (1 - rho_s/rho_l) d f_s/dt, previous  */
    LBM_FIELD_Q_PREV = 6,   /* rho C_p T mdot, previous step                     */
    LBM_FIELD_PSIUX = 7,    /* psi u_x of the previous step (Euler d_t(psi u))   */
    LBM_FIELD_PSIUY = 8,    /* psi u_y of the previous step                      */
    LBM_FIELD_P = 9,        /* pressure p of the previous step                   */
    LBM_FIELD_S = 10,       /* S = rho mdot + u . grad rho of the previous step  */
    LBM_FIELD_PSI = 11,     /* order parameter psi at time n        (read only)  */
    LBM_FIELD_FSOLID = 12,  /* solid fraction f_s at time n         (read only)  */
    LBM_FIELD_T = 13,       /* temperature T at time n              (read only)  */
    LBM_FIELD_PHI = 14,     /* electric potential phi at time n     (read only)  */
    LBM_FIELD_HTOT = 15,    /* total enthalpy H at time n           (read only)  */
    LBM_FIELD_SIGMA = 16    /* conductivity used by the extra potential sweeps   */
};

/* Message of the last failing call on this thread (static storage). */
const char *lbm_last_error(void);

/*
 * Create an instance.  Validates `p` (see lbm_params), derives the lattice
 * constants of Secs. 2-3, and allocates the device state: ONE copy of the
 * 32 populations per cell (f 9, h 9, g 9, l 5) in the precision's storage
 * type, streamed in place (AA pattern: the layout alternates between steps),
 * two copies of 7 per-cell auxiliary fields (previous-step f_s, mdot,
 * rho C_p T mdot, psi u_x, psi u_y, p, S), sigma, a record of
 * (psi, f_s, phi) per cell in the arithmetic type (each step stores those
 * of the tile-edge cells first, for their neighbour tiles' halos) and a
 * small reduction workspace: about 204 bytes per cell in FP32, 158 in
 * LBM_FP16S, 408 in FP64.  `stream` is a cudaStream_t (NULL: the legacy
 * default stream); all work of the handle is enqueued there.
 * On success *out owns the memory until lbm_destroy.
 * Errors: BADPARAM, OOM, CUDA.
 */
int lbm_create(const lbm_params *p, void *stream, struct lbm_handle **out);

/*
 * Initial state (Sec. 2; Algorithm 1 "Initialization"): a circular droplet
 * of radius R centred at (xc, yc) in cell coordinates (cell (x, y) sits at
 * (x, y); the bottom wall is y = -1/2), psi = 1/2 + 1/2 tanh(2 (R - r) / W);
 * fluid at rest, p = 0, T = T_init, no solid, all latent heat held
 * (H = C_p T + psi L); phi linear between the electrodes; every population
 * at its equilibrium.  Then `presolve` sweeps of the potential LB relax phi
 * around the droplet before t = 0 (the field and the cold wall act from
 * t = 0, Sec. 2).  A sessile cap at contact angle theta has
 * yc = -1/2 - R cos(theta).  Resets the step counter and t_fre.
 * Errors: BADPARAM (R <= 0, presolve < 0), CUDA.
 */
int lbm_init_droplet(struct lbm_handle *h, double R, double xc, double yc, int32_t presolve);

/*
 * Same initial state from an arbitrary order-parameter field: `psi` is a
 * host array of ny * nx doubles (row-major, x fastest), copied during the
 * call.  Errors: BADPARAM (NULL psi, presolve < 0), CUDA.
 */
int lbm_init_psi(struct lbm_handle *h, const double *psi, int32_t presolve);

/*
 * Pre-solve of the potential to a tolerance (Algorithm 1's convergence of
 * the electric field before the coupled run; reading R15): potential sweeps
 * with sigma and every other field frozen, until the largest change of phi
 * over one sweep, relative to |phi_top - phi_bot|, is below tol; measured
 * every 64 sweeps, at most max_sweeps in all.  *sweeps and *residual (each
 * may be NULL) receive the sweeps run and the last measured change.  The
 * same sweeps as lbm_init_*'s `presolve` count: an init with presolve =
 * *sweeps reaches the same state.  In half storage the sweeps round
 * stochastically, which leaves a per-sweep change of a few 1e-4 of the
 * electrode difference: tighter tolerances end at max_sweeps with the
 * warning (the field itself settles to about 2e-4 of that difference).
 * Synchronises the stream.  Returns LBM_OK,
 * LBM_WARN_NOT_CONVERGED (> 0) when max_sweeps ran out first, or BADPARAM
 * (NULL handle, tol <= 0, max_sweeps < 1), STATE (before init), DIVERGED
 * (non-finite potential), CUDA.
 */
int lbm_presolve(struct lbm_handle *h, double tol, int32_t max_sweeps, int32_t *sweeps, double *residual);

/*
 * Advance n >= 0 time steps (Algorithm 1 under a Jacobi reading: every
 * system collides with time-n fields, then all stream, then the walls act).
 * Each step is two launches over the lattice (the halo records of the
 * tile-edge cells, then the fused step, streaming in place), plus k_e - 1
 * potential-only sweeps (sigma frozen at time n).  Enqueues asynchronously
 * on the handle's stream (long runs replay a captured CUDA graph).
 * Errors: STATE (not initialised), DIVERGED (an earlier observables call
 * saw non-finite values), BADPARAM (n < 0), CUDA.
 */
int lbm_step(struct lbm_handle *h, int64_t n);

/*
 * Observables at the current time (see lbm_obs), reduced on the GPU (FP64
 * above the first, 32-cell level) and copied to *out.  Synchronises the stream.  Updates t_fre.
 * Returns LBM_ERR_DIVERGED (and sets out->status) if a non-finite psi or H
 * was found.  Errors: BADPARAM (NULL out), STATE, CUDA.
 */
int lbm_observables(struct lbm_handle *h, lbm_obs *out);

/*
 * Enqueue the observables reduction without waiting; the result stays on
 * the device until lbm_observables_fetch copies it (synchronising).
 * Errors: STATE, CUDA.
 */
int lbm_observables_async(struct lbm_handle *h);
int lbm_observables_fetch(struct lbm_handle *h, lbm_obs *out);

/*
 * Streaming observables: enqueue the reduction of lbm_observables (Secs.
 * 4-5) and the copy of its result into the caller's host memory *out on the
 * handle's stream, and return without waiting.  With *out in page-locked memory the copy is
 * asynchronous, so a loop of steps and observations runs without a host
 * round trip per step; *out holds the values once lbm_sync has returned and
 * must stay valid until then (pageable memory works too, the copy then
 * waits).  Divergence is reported in out->status (LBM_ERR_DIVERGED), not by
 * the return value, and does not stop later steps.  Errors: BADPARAM (NULL),
 * STATE, CUDA.
 */
int lbm_observables_to_host(struct lbm_handle *h, lbm_obs *out);

/*
 * Observation fused into the next step: request the observables of the
 * current state (those of lbm_observables, Secs. 4-5) without a pass of
 * their own over the lattice.  The next
 * lbm_step reduces them inside its first step's kernel, which reads exactly
 * this state (its macro, stencil and force stages evaluate every value they
 * need), and a small finish launch after it sums the kernel's block
 * partials; any other call on the handle first runs them on their own, as
 * lbm_observables_async would.  out: NULL to fetch the result later with
 * lbm_observables_fetch, or host memory (page-locked for an asynchronous
 * copy) that receives it behind that kernel, as lbm_observables_to_host.
 * Same values as lbm_observables at this step, up to the grouping of the
 * FP64 sums (the step's tiles are 32 x tile_rows, the observables kernel's
 * 32 x 8).
 * Errors: BADPARAM (NULL handle), STATE, CUDA.
 */
int lbm_observables_deferred(struct lbm_handle *h, lbm_obs *out);

/*
 * Wait for everything enqueued on the handle's stream (running a deferred
 * observation first).  Returns CUDA if a bounded wait inside a step kernel
 * ran out (the status lbm_observables reports).  Errors: BADPARAM (NULL),
 * CUDA.
 */
int lbm_sync(struct lbm_handle *h);

/*
 * Copy one field to the host as doubles (layout: see the field ids).
 * Synchronises the stream.  Errors: BADPARAM (unknown id, NULL), STATE, CUDA.
 */
int lbm_get_field(struct lbm_handle *h, int32_t field, double *host_out);

/*
 * Overwrite one stored field (ids 0-10 and 16) from host doubles, converting
 * to the storage precision.  Synchronises.  Errors: BADPARAM (read-only id,
 * NULL), STATE, CUDA.
 */
int lbm_set_field(struct lbm_handle *h, int32_t field, const double *host_in);

/*
 * Whole-state snapshot for checkpoint/resume and host hand-over: the step
 * counter, the stochastic-rounding counter, t_fre and every stored array in
 * the handle's storage precision, populations always in the natural layout
 * (population i of cell (x, y) in plane i at (x, y), whatever the layout
 * phase of the in-place streaming; export converts on the host).  The
 * header records the layout phase the state was in, and import restores
 * the state into that phase on the device, so a resumed run takes the same
 * step kernels as the original and reproduces it bit for bit.
 * lbm_state_bytes gives the size; export copies device -> host (synchronous),
 * import copies host -> device and is ordered on the handle's stream: the
 * whole snapshot goes into one of two device buffers on a private copy
 * stream, which does not wait for the work already enqueued on the handle's
 * stream, and the handle's stream then unpacks it (device to device).  From
 * pinned host memory the call is asynchronous: the caller keeps the buffer
 * alive and unchanged until the handle's stream has passed the import (for
 * instance lbm_sync).  The first import allocates the two buffers
 * (2 x lbm_state_bytes of device memory, kept until lbm_destroy).  A
 * snapshot only imports into a handle created with identical lbm_params.
 * Errors: BADPARAM (NULL, size mismatch), OOM, STATE, CUDA.
 */
size_t lbm_state_bytes(const struct lbm_handle *h);
int lbm_export_state(struct lbm_handle *h, void *host, size_t bytes);
int lbm_import_state(struct lbm_handle *h, const void *host, size_t bytes);

/*
 * Step kernel selection (tuning and testing; results do not depend on it in
 * FP64, and differ only by rounding in FP32).  Every step is two launches:
 * the halo records of the tile-edge cells, then the step kernel:
 *   variant LBM_STEP_DIRECT (the one variant): one block per tile; every
 *     thread copies its cell's populations into shared memory for the
 *     collisions;
 *   tile_rows: 4, 8 or 16 lattice rows per 32-column tile (default 4 in
 *     single precision, 8 in FP64).
 * Errors: BADPARAM (unknown variant or height, NULL).
 */
enum { LBM_STEP_DIRECT = 1 };
int lbm_configure(struct lbm_handle *h, int32_t variant, int32_t tile_rows);

/*
 * Observables of a caller-held state, allocating nothing.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, such as code
 * embedded in a runtime that has already reserved the device memory for its
 * own pool, or a latency-critical loop in which an allocation would
 * synchronise the device.  It runs the same reduction as lbm_observables
 * with its scratch (block partial sums, crossing candidates) in a
 * fixed-size array that the library keeps in device memory on every GPU
 * that loads it (about 1.3 MB, held until the process exits).
 *   p     parameters of the state (host struct, read during the call)
 *   pop   device array of 32 planes, f 0-8 then h 0-8, g 0-8, l 0-4, in the
 *         natural layout (population i of cell (x, y) in plane i), each
 *         ny rows of `pitch` elements, x fastest: all in double for
 *         LBM_FP64, all in float for LBM_FP32; for LBM_FP16S the 9 f planes
 *         in float followed by the 23 others in half -- for example the body
 *         of an lbm_export_state snapshot after its 64-byte header (pitch =
 *         nx rounded up to 32)
 *   aux   device array of the 7 auxiliary planes that follow `pop` in such a
 *         snapshot (FP64 for LBM_FP64, else FP32), same plane layout
 *   pitch elements per row (>= nx); step: step number reported in out
 *   out   device lbm_obs written by the call; its t_fre is read and kept, so
 *         set t_fre = -1 before the first call on a run
 *   stream cudaStream_t on which the work is enqueued (the call returns
 *         without waiting; synchronise before reading out)
 * Limits: ny <= 4096 and at most 20480 tiles of 32 x 8 cells (about 5.2
 * million cells); larger lattices return LBM_ERR_BADPARAM.  pop and aux
 * must be aligned to their element size (8 bytes for LBM_FP64, 4 otherwise)
 * and out to 8 bytes, else LBM_ERR_BADPARAM.
 * A call looks up the array's device address on the current device (a
 * device reset moves it); a call made while `stream` is being captured uses
 * the address of the last lookup on that device instead, so make one call
 * before any stream capture (a capture before it returns LBM_ERR_CUDA).
 * Every call shares the one array and clears what must start at zero, so
 * calls whose work overlaps on the GPU (several streams at once) race;
 * serialise them.  Errors: BADPARAM (NULL pointers, invalid parameters,
 * size limits, misaligned pointers), CUDA (lookup or launch failure).
 */
int lbm_observables_noalloc(const lbm_params *p, const void *pop, const void *aux, int32_t pitch,
                            int64_t step, lbm_obs *out, void *stream);

/*
 * Local heat flux through the cold substrate (Sec. 4.3): Fourier's law with
 * the one-sided second-order difference over the first three cell rows,
 *   host_out[x] = -k(x,0) (4 T(x,1) - T(x,2) - 3 T(x,0)) / 2,
 * k the local conductivity of row 0 (rho C_p alpha mixed by phase), in the
 * handle's arithmetic precision, returned as nx host doubles.  Negative
 * where heat flows into the cold wall.  Synchronises the handle's stream.
 * Errors: BADPARAM (NULL, ny < 3), STATE (before init), CUDA.
 */
int lbm_substrate_heat_flux(struct lbm_handle *h, double *host_out);

/*
 * The stochastic rounding of half storage (LBM_FP16S, Sec. 3's populations
 * g and l kept as weight-shifted halves), exposed so that the conversion
 * the step uses can be checked against its definition: out[i] receives the
 * 16 bits of v[i] rounded to half with the 13 random bits r[i] & 0x1fff
 * (the step draws them from Philox4x32-10; here the caller supplies them).
 *   |v| in the normal half range [2^-14, 65504]: with s the half spacing at
 *     |v| and d the 13 bits of |v| below it (|v| = (q + d / 2^13) s, q an
 *     integer), the magnitude is (q + 1) s if d + r >= 2^13, else q s;
 *   |v| < 2^-14 (subnormal halves, spacing 2^-24): |v| + r 2^-37, rounded
 *     to single precision, truncated to a multiple of 2^-24;
 *   beyond the half range: the largest finite half, 65504; the sign is
 *     kept; NaN stays NaN.
 * So over the 8192 values of r the mean of the normal-range result is v
 * exactly: the rounding is unbiased.
 *   v, r, out  device arrays of n elements (v float, 4-byte aligned; r
 *              uint32, 4-byte aligned; out uint16, 2-byte aligned), owned
 *              by the caller
 *   stream     cudaStream_t on which the work is enqueued (the call returns
 *              without waiting)
 * Errors: BADPARAM (n < 0, NULL or misaligned pointers with n > 0), CUDA
 * (launch failure).  n = 0 enqueues nothing.
 */
int lbm_round_half_sr(const float *v, const uint32_t *r, uint16_t *out, int64_t n, void *stream);

/* Steps taken since the last init.  */
int64_t lbm_step_count(const struct lbm_handle *h);

/* Device memory the handle holds, in bytes: the state allocated by
 * lbm_create (see there) and the reduction workspace, plus the field
 * staging buffer and the two import buffers once a call has allocated them.
 * 0 for NULL. */
size_t lbm_device_bytes(const struct lbm_handle *h);

/* Free the device state.  NULL is ignored. */
void lbm_destroy(struct lbm_handle *h);

/*
 * Batched form: many instances of one precision advance together, one
 * persistent kernel launch per time step over a work list of (instance,
 * tile) pairs, so small and uneven lattices fill the GPU.  Members stay
 * owned by the caller, keep their own state and stay usable alone (their
 * results are the same as stepping them one by one); the batch holds only
 * the work list and its launch configuration.  Every member must be
 * initialised, share the precision, and use the stream the batch was given.
 * tile_rows picks the tile height (0: autotuned once at creation by timing
 * the candidate shapes on the members).
 * Errors: BADPARAM (n < 1, mixed precision, NULL), STATE, OOM, CUDA.
 */
int lbm_batch_create(struct lbm_handle *const *members, int32_t n, void *stream,
                     int32_t tile_rows, struct lbm_batch **out);
int lbm_batch_step(struct lbm_batch *b, int64_t n);
int32_t lbm_batch_tile_rows(const struct lbm_batch *b);
void lbm_batch_destroy(struct lbm_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
