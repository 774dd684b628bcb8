// Host side of the C ABI declared in include/lbm.h: parameter validation,
// derived lattice constants, device memory, stepping (with CUDA-graph
// replay of long runs), observables, field access, snapshots and batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t storage_bytes(int precision) {
    return precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2);
}
size_t aux_bytes(int precision) { return precision == LBM_FP64 ? 8 : 4; }
// Population copy layout: 9 f planes, then h, g, l (9, 9, 5 planes) of the
// storage type; half storage keeps f in single precision.
size_t f_bytes(int precision) { return precision == LBM_FP64 ? 8 : 4; }
size_t pop_cell_bytes(int precision) { return 9 * f_bytes(precision) + (NPOP - 9) * storage_bytes(precision); }
size_t l_offset_bytes(int precision, long long plane) {
    return (size_t)plane * (9 * f_bytes(precision) + 18 * storage_bytes(precision));
}
// Halo record of a tile-edge cell: (psi, f_s, phi) and a pad, in the
// arithmetic type (FP32 16 bytes, FP64 32).
size_t halo_rec_bytes(int precision) { return precision == LBM_FP64 ? 32 : 16; }

// D2Q9 and D2Q5 velocity sets (Secs. 3.1, 3.4) for the host-side layout
// conversion of snapshots.
const int HCX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, HCY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const int HOPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
const int HCX5[5] = {0, 1, 0, -1, 0}, HCY5[5] = {0, 0, 1, 0, -1}, HOPP5[5] = {0, 3, 4, 1, 2};

// Rewrite nq planes of elements of `es` bytes, held in the swapped layout of
// the in-place streaming (population i of cell x in plane opp(i) at x - c_i,
// or in plane i at x where x - c_i lies beyond a wall), into the natural one
// (population i of cell x in plane i at x).
void unswap_planes(char *buf, size_t es, int nq, int nx, int ny, int pitch, long long plane) {
    const int *cx = nq == 9 ? HCX : HCX5, *cy = nq == 9 ? HCY : HCY5, *op = nq == 9 ? HOPP9 : HOPP5;
    std::vector<char> raw(buf, buf + (size_t)nq * plane * es);
    for (int i = 0; i < nq; i++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                const int yu = y - cy[i];
                int q = i, sy = y, sx = x;
                if (yu >= 0 && yu < ny && (cx[i] != 0 || cy[i] != 0)) {
                    q = op[i];
                    sy = yu;
                    sx = ((x - cx[i]) % nx + nx) % nx;
                }
                std::memcpy(buf + ((size_t)i * plane + (size_t)y * pitch + x) * es,
                            raw.data() + ((size_t)q * plane + (size_t)sy * pitch + sx) * es, es);
            }
}

// Lattice constants from the dimensionless parameters (Secs. 2-4).
void derive(const lbm_params &p, Consts<double> &c) {
    c.rho[1] = p.rho_l;
    c.rho[2] = p.rho_l / p.rho_lg;
    c.rho[0] = p.rho_l * p.rho_sl;
    c.mu[1] = p.mu_l;
    c.mu[2] = p.mu_l / p.mu_lg;
    c.mu[0] = p.mu_l;
    c.cp[0] = p.cp_s;
    c.cp[1] = p.cp_l;
    c.cp[2] = p.cp_g;
    c.kth[1] = c.rho[1] * c.cp[1] * p.alpha_l;                  // k = rho C_p alpha
    c.kth[2] = c.rho[2] * c.cp[2] * (p.alpha_l / p.alpha_lg);
    c.kth[0] = c.rho[0] * c.cp[0] * (p.alpha_l * p.alpha_sl);   // alpha_s = alpha_l alpha_sl
    c.eps[2] = p.eps_g;
    c.eps[1] = p.S_eps * p.eps_g;
    c.eps[0] = c.eps[1];
    c.sig[2] = p.sigma_g;
    c.sig[1] = p.R_sigma * p.sigma_g;
    c.sig[0] = c.sig[1];
    c.L = p.cp_l * (p.T_m - p.T_w) / p.Ste;
    c.Cref = 2.0 * p.cp_s * p.cp_l / (p.cp_s + p.cp_l);
    c.kappa = 1.5 * p.gamma * p.W;
    c.beta = 12.0 * p.gamma / p.W;
    c.tau_f = p.M / (1.0 / 3.0) + 0.5;
    const double E0 = std::sqrt(p.CaE * p.gamma / (p.eps_g * p.R0));
    c.phi_bot = 0.0;
    c.phi_top = E0 * p.ny;
    c.wet = 4.0 / p.W * std::cos(p.theta_deg * 3.14159265358979323846 / 180.0);
    c.T_m = p.T_m;
    c.W = p.W;
    c.one_m_rsl = 1.0 - c.rho[0] / c.rho[1];
    c.Cref_Tw = c.Cref * p.T_w;
    c.T_init = p.T_init;
    c.om_f = 1.0 / c.tau_f;
    c.pre_f = 1.0 - 0.5 / c.tau_f;
    c.four_over_W = 4.0 / p.W;
    c.three_over_Cref = 3.0 / c.Cref;          // 1 / (C_p,ref c_s^2)
}

template <typename T>
Consts<T> cast_consts(const Consts<double> &d) {
    Consts<T> c;
    for (int i = 0; i < 3; i++) {
        c.rho[i] = T(d.rho[i]);
        c.mu[i] = T(d.mu[i]);
        c.kth[i] = T(d.kth[i]);
        c.cp[i] = T(d.cp[i]);
        c.eps[i] = T(d.eps[i]);
        c.sig[i] = T(d.sig[i]);
    }
    c.L = T(d.L); c.Cref = T(d.Cref); c.kappa = T(d.kappa); c.beta = T(d.beta);
    c.tau_f = T(d.tau_f); c.phi_bot = T(d.phi_bot); c.phi_top = T(d.phi_top); c.wet = T(d.wet);
    c.T_m = T(d.T_m); c.W = T(d.W); c.one_m_rsl = T(d.one_m_rsl); c.Cref_Tw = T(d.Cref_Tw);
    c.T_init = T(d.T_init);
    c.om_f = T(d.om_f); c.pre_f = T(d.pre_f); c.four_over_W = T(d.four_over_W);
    c.three_over_Cref = T(d.three_over_Cref);
    return c;
}

bool pos(double v) { return v > 0.0; }   // false for NaN

const char *validate(const lbm_params &p) {
    if (p.nx <= 0 || p.ny <= 0) return "nx and ny must be positive";
    // the step kernels address a cell's planes with 32-bit offsets
    if ((uint64_t)NPOP * (uint64_t)((p.nx + 31) / 32 * 32) * (uint64_t)p.ny > 0xFFFFFFFFull)
        return "lattice too large: 32 x (nx rounded up to 32) x ny must stay below 2^32 elements";
    if ((long long)p.nx * p.ny > (1LL << 28)) return "lattice too large";
    if (p.k_e < 1) return "k_e must be >= 1";
    if (p.precision < LBM_FP64 || p.precision > LBM_FP16S) return "unknown precision";
    if (!pos(p.W) || !pos(p.M)) return "W and M must be positive";
    if (!(p.gamma >= 0.0) || !(p.CaE >= 0.0)) return "gamma and CaE must be >= 0";
    if (!pos(p.rho_l) || !pos(p.rho_lg) || !pos(p.rho_sl)) return "densities must be positive";
    if (!pos(p.mu_l) || !pos(p.mu_lg)) return "viscosities must be positive";
    if (!pos(p.Ste) || !pos(p.alpha_l) || !pos(p.alpha_lg) || !pos(p.alpha_sl))
        return "Ste and diffusivities must be positive";
    if (!pos(p.cp_l) || !pos(p.cp_s) || !pos(p.cp_g)) return "heat capacities must be positive";
    if (!pos(p.R_sigma) || !pos(p.S_eps) || !pos(p.eps_g) || !pos(p.sigma_g)) return "electric properties must be positive";
    if (!pos(p.R0)) return "R0 must be positive";
    if (!(p.theta_deg > 0.0 && p.theta_deg < 180.0)) return "theta must lie in (0, 180)";
    if (!(p.T_m >= p.T_w)) return "T_m must be >= T_w";
    if (!std::isfinite(p.T_init)) return "T_init must be finite";
    return nullptr;
}

// Half-precision storage references and scales (weight-shifted form):
//   f_i stored as f_i - w_i          (zero in the liquid, -w_i in the gas)
//   h_i stored as 2^10 h_i           (h ~ w_i p / c_s^2, keeps it normal in half)
//   g_i stored as g_i - w_i C_p,ref T_m (i > 0) and g_0 - (L/2 - (1 - w_0) C_p,ref T_m)
//                                    (the rest population spans the latent heat)
//   l_i stored as (l_i - l_eq,i(phi_lin(y))) * 2^k, 2^k ~ 1 / E0
//                                    (deviation from the uniform field)
// Powers of two keep the scaling exact.
Shift make_shift(const lbm_params &p, const Consts<double> &c) {
    Shift s;
    s.f_ref = 1.0f;
    // g: the equilibria of liquid at rest at the melting point (g_0 =
    // H - C_p,ref T + w_0 C_p,ref T with H = C_p,l T_m + L).  The liquid
    // then stores values near zero, where half precision is finest: there
    // T sits at T_m and H performs an undamped walk under rounding noise
    // (latent-heat plateau), while in ice and gas conduction damps it.
    s.g_ref = float(c.Cref * p.T_m);
    s.g0_ref = float(c.L + p.cp_l * p.T_m - c.Cref * p.T_m + (4.0 / 9.0) * c.Cref * p.T_m);
    s.h_scale = 1024.0f;
    const double E0 = (c.phi_top - c.phi_bot) / p.ny;
    s.l_scale = E0 > 1e-12 ? (float)std::exp2(std::round(std::log2(1.0 / E0))) : 1.0f;
    s.f_scale = 1.0f;
    s.g_scale = 1.0f;
    return s;
}

int obs_grid_blocks(int nx, int ny) { return ((nx + 31) / 32) * ((ny + 7) / 8); }

}  // namespace

int lbm::obs_blocks(int nx, int ny) { return obs_grid_blocks(nx, ny); }

void lbm::set_last_error(const std::string &msg) { g_err = msg; }

// Validation and derived constants for entry points that hold no handle.
int lbm::derive_for_noalloc(const lbm_params *p, Consts<double> *cd, Consts<float> *cf, Shift *sh,
                            const char **why) {
    if (const char *w = validate(*p)) {
        *why = w;
        return LBM_ERR_BADPARAM;
    }
    derive(*p, *cd);
    *cf = cast_consts<float>(*cd);
    *sh = make_shift(*p, *cd);
    return LBM_OK;
}

struct lbm_handle {
    lbm_params P;
    Consts<double> cd;
    Consts<float> cf;
    Shift sh;
    DevState s;
    cudaStream_t st;
    cudaStream_t cap;          // private stream used only to capture graphs
    void *mem = nullptr;
    size_t mem_bytes = 0;
    void *ws_mem = nullptr;
    size_t ws_mem_bytes = 0;
    ObsScratch ws;
    size_t ws_max_bytes = 0, ws_min_bytes = 0, ws_u32_bytes = 0;
    unsigned long long *ws_max_base = nullptr, *ws_min_base = nullptr;
    unsigned int *ws_u32_base = nullptr;
    double *staging = nullptr;
    // two device copies of imported snapshots: the host-to-device copy of an
    // import runs on its own stream while the handle's stream still works
    // on the state before it (allocated by the first import)
    void *imp_buf[2] = {nullptr, nullptr};
    cudaStream_t imp_st = nullptr;
    cudaEvent_t imp_filled[2] = {nullptr, nullptr}, imp_free[2] = {nullptr, nullptr};
    int imp_next = 0;
    uint32_t presolve_sweeps = 0;    // pre-solve sweeps run so far (rounding streams)
    // an observation requested and not yet run: the next lbm_step runs it
    // inside its first step's kernel (the state it reads is the one
    // observed); any other call runs it first on its own
    bool obs_pending = false;
    Scalars obs_sc;
    lbm_obs *obs_out = nullptr;      // host copy requested with it, if any
    int cur = 0, lcur = 0;
    int64_t step = 0;
    bool inited = false, diverged = false;
    int tile_rows = 4;         // lattice rows per tile (set per precision in lbm_create)
    int variant = LBM_STEP_DIRECT;   // form of the step kernel (lbm_configure)
    unsigned int *err = nullptr;   // device status word (sticky error bits)
    double *qdot = nullptr;        // nx doubles: substrate heat flux profile
    // graph cache: one per starting parity (cur, lcur)
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int gsteps = 0;
};

// A device work list of (member, tile) pairs with its launch shape and a
// graph cache per starting parity.
struct WorkList {
    BatchItem *items_dev = nullptr;
    void *consts_dev = nullptr;
    int *tile_item_dev = nullptr;      // member of every step tile
    int n = 0;
    int total_tiles = 0, total_sweep_tiles = 0, grid = 0, sweep_grid = 0;
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
};

struct lbm_batch {
    std::vector<lbm_handle *> m;
    int precision = LBM_FP32;
    int k_e = 1;
    int tile_rows = 8;
    cudaStream_t st = nullptr;
    WorkList all;                  // every member: one launch per step
    std::vector<WorkList> groups;  // members grouped so each group's state fits in L2
    int flips = 0;                 // steps since the lists were built (mod 2 matters)
    int lflips = 0;                // potential sweeps since then
    std::vector<int> cur0, lcur0;  // member parities when the lists were built
    cudaStream_t cap = nullptr;    // private capture stream
};

namespace {

const void *consts_for(const lbm_handle *h) {
    return h->P.precision == LBM_FP64 ? static_cast<const void *>(&h->cd) : static_cast<const void *>(&h->cf);
}

cudaError_t do_step(lbm_handle *h, cudaStream_t st, const Scalars *observe = nullptr) {
    const int ws = h->P.k_e > 1 ? 1 : 0;
    const void *c = consts_for(h);
    cudaError_t e;
    if (observe) {           // the step also reduces the observables of the state it reads
        switch (h->P.precision) {
        case LBM_FP64: e = launch_step_obs_f64(h->s, h->cur, h->lcur, ws, c, h->sh, h->tile_rows, h->ws, *observe, st); break;
        case LBM_FP32: e = launch_step_obs_f32(h->s, h->cur, h->lcur, ws, c, h->sh, h->tile_rows, h->ws, *observe, st); break;
        default: e = launch_step_obs_f16s(h->s, h->cur, h->lcur, ws, c, h->sh, h->tile_rows, h->ws, *observe, st); break;
        }
    } else {
        switch (h->P.precision) {
        case LBM_FP64: e = launch_step_f64(h->s, h->cur, h->lcur, ws, c, h->sh, h->tile_rows, h->variant, st); break;
        case LBM_FP32: e = launch_step_f32(h->s, h->cur, h->lcur, ws, c, h->sh, h->tile_rows, h->variant, st); break;
        default: e = launch_step_f16s(h->s, h->cur, h->lcur, ws, c, h->sh, h->tile_rows, h->variant, st); break;
        }
    }
    if (e != cudaSuccess) return e;
    h->cur ^= 1;
    h->lcur ^= 1;
    // the extra sweeps round with the next step's counter, on streams 4, 5, ...
    // (the step itself uses 0-3)
    for (int j = 1; j < h->P.k_e; j++) {
        const uint32_t sys = 3u + (uint32_t)j;
        switch (h->P.precision) {
        case LBM_FP64: e = launch_sweep_f64(h->s, h->lcur, h->cur, sys, c, h->sh, st); break;
        case LBM_FP32: e = launch_sweep_f32(h->s, h->lcur, h->cur, sys, c, h->sh, st); break;
        default: e = launch_sweep_f16s(h->s, h->lcur, h->cur, sys, c, h->sh, st); break;
        }
        if (e != cudaSuccess) return e;
        h->lcur ^= 1;
    }
    return cudaSuccess;
}

// A pre-solve sweep: its rounding stream (half storage) is the handle's
// running count of pre-solve sweeps with the top bit set, apart from the
// streams of the steps.
cudaError_t do_sweep(lbm_handle *h, cudaStream_t st) {
    const void *c = consts_for(h);
    const uint32_t sys = 0x80000000u | (h->presolve_sweeps++ & 0x7fffffffu);
    cudaError_t e;
    switch (h->P.precision) {
    case LBM_FP64: e = launch_sweep_f64(h->s, h->lcur, h->cur, sys, c, h->sh, st); break;
    case LBM_FP32: e = launch_sweep_f32(h->s, h->lcur, h->cur, sys, c, h->sh, st); break;
    default: e = launch_sweep_f16s(h->s, h->lcur, h->cur, sys, c, h->sh, st); break;
    }
    if (e == cudaSuccess) h->lcur ^= 1;
    return e;
}

// Run a pending observation on its own (the observables kernel) and the
// host copy requested with it; every entry point that reads or changes the
// state, other than lbm_step, calls this first.
int run_pending_obs(lbm_handle *h) {
    if (!h->obs_pending) return LBM_OK;
    h->obs_pending = false;
    cudaError_t e;
    switch (h->P.precision) {
    case LBM_FP64: e = launch_obs_f64(h->s, h->cur, h->lcur, &h->cd, h->sh, h->ws, h->obs_sc, h->st); break;
    case LBM_FP32: e = launch_obs_f32(h->s, h->cur, h->lcur, &h->cf, h->sh, h->ws, h->obs_sc, h->st); break;
    default: e = launch_obs_f16s(h->s, h->cur, h->lcur, &h->cf, h->sh, h->ws, h->obs_sc, h->st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "observables kernels");
    if (h->obs_out) {
        lbm_obs *out = h->obs_out;
        h->obs_out = nullptr;
        CK(cudaMemcpyAsync(out, h->ws.obs, sizeof(lbm_obs), cudaMemcpyDeviceToHost, h->st));
    }
    return LBM_OK;
}

void drop_graphs(lbm_handle *h) {
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            if (h->gexec[a][b]) {
                cudaGraphExecDestroy(h->gexec[a][b]);
                h->gexec[a][b] = nullptr;
            }
}

int ensure_staging(lbm_handle *h) {
    if (h->staging) return LBM_OK;
    const size_t n = (size_t)9 * h->P.nx * h->P.ny;
    if (cudaMalloc(&h->staging, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        h->staging = nullptr;
        return fail(LBM_ERR_OOM, "staging allocation failed");
    }
    return LBM_OK;
}

int finish_init(lbm_handle *h, const double *psi_dev, double R, double xc, double yc, int presolve) {
    if (int rc_ = run_pending_obs(h)) return rc_;
    h->cur = 0;
    h->lcur = 0;
    const void *c = consts_for(h);
    cudaError_t e;
    switch (h->P.precision) {
    case LBM_FP64: e = launch_init_f64(h->s, psi_dev, R, xc, yc, c, h->sh, h->st); break;
    case LBM_FP32: e = launch_init_f32(h->s, psi_dev, R, xc, yc, c, h->sh, h->st); break;
    default: e = launch_init_f16s(h->s, psi_dev, R, xc, yc, c, h->sh, h->st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    for (int j = 0; j < presolve; j++) {
        e = do_sweep(h, h->st);
        if (e != cudaSuccess) return cuda_fail(e, "pre-solve sweep");
    }
    lbm_obs o;
    std::memset(&o, 0, sizeof o);
    o.t_fre = -1;
    o.Fo_fre = -1.0;
    CK(cudaMemcpyAsync(h->ws.obs, &o, sizeof o, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->step = 0;
    h->inited = true;
    h->diverged = false;
    return LBM_OK;
}

}  // namespace

extern "C" {

const char *lbm_last_error(void) { return g_err.c_str(); }

int lbm_create(const lbm_params *p, void *stream, lbm_handle **out) {
    if (!p || !out) return fail(LBM_ERR_BADPARAM, "NULL argument");
    *out = nullptr;
    if (const char *why = validate(*p)) return fail(LBM_ERR_BADPARAM, why);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(LBM_ERR_CUDA, "no CUDA device");
    }
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return fail(LBM_ERR_OOM, "host allocation failed");
    h->P = *p;
    // measured on GB300 at 512 x 256: per-thread loads with 4-row tiles are
    // the fastest single-precision form; FP64 (arithmetic-bound) uses 8 rows
    h->tile_rows = p->precision == LBM_FP64 ? 8 : 4;
    derive(*p, h->cd);
    h->cf = cast_consts<float>(h->cd);
    h->sh = make_shift(*p, h->cd);
    h->st = static_cast<cudaStream_t>(stream);
    const int nx = p->nx, ny = p->ny;
    const int pitch = (int)round_up(nx, 32);
    const long long plane = (long long)pitch * ny;
    const size_t sb = storage_bytes(p->precision), ab = aux_bytes(p->precision);
    const size_t pop_b = round_up((size_t)plane * pop_cell_bytes(p->precision), 256);
    (void)sb;
    const size_t aux_b = round_up((size_t)NAUX * plane * ab, 256);
    const size_t sig_b = round_up((size_t)plane * ab, 256);
    const size_t halo_b = round_up((size_t)plane * halo_rec_bytes(p->precision), 256);
    // one population copy: the step streams in place (AA pattern)
    h->mem_bytes = pop_b + 2 * aux_b + sig_b + halo_b;
    if (cudaMalloc(&h->mem, h->mem_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(LBM_ERR_OOM, "device allocation of the state failed");
    }
    char *b = static_cast<char *>(h->mem);
    h->s.pop = b;
    h->s.aux[0] = b + pop_b;
    h->s.aux[1] = b + pop_b + aux_b;
    h->s.sigma = b + pop_b + 2 * aux_b;
    h->s.halo = b + pop_b + 2 * aux_b + sig_b;
    h->s.nx = nx;
    h->s.ny = ny;
    h->s.pitch = pitch;
    h->s.plane = plane;
    // observables workspace
    // sized for the larger grid: the observables kernel's or, for the
    // observation fused into a step, the step's with 4-row tiles
    const int nb = std::max(obs_grid_blocks(nx, ny), ((nx + 31) / 32) * ((ny + 3) / 4));
    const int ng = (nb + OBS_GROUP - 1) / OBS_GROUP;
    const size_t part_b = round_up((size_t)(nb + ng) * OBS_NSUM * sizeof(double), 256);
    const size_t qdot_b = round_up((size_t)nx * sizeof(double), 256);
    h->ws_max_bytes = round_up((size_t)(2 + ny) * 8, 256);
    h->ws_min_bytes = round_up((size_t)(1 + ny) * 8, 256);
    h->ws_u32_bytes = round_up((size_t)(ny + 3 + ng) * 4, 256);
    const size_t obs_b = round_up(sizeof(lbm_obs), 256);
    const size_t err_b = 256;
    h->ws_mem_bytes = part_b + h->ws_max_bytes + h->ws_min_bytes + h->ws_u32_bytes + obs_b + err_b + qdot_b;
    if (cudaMalloc(&h->ws_mem, h->ws_mem_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->mem);
        delete h;
        return fail(LBM_ERR_OOM, "device allocation of the reduction workspace failed");
    }
    char *w = static_cast<char *>(h->ws_mem);
    h->ws.partials = reinterpret_cast<double *>(w);
    h->ws_max_base = reinterpret_cast<unsigned long long *>(w + part_b);
    h->ws_min_base = reinterpret_cast<unsigned long long *>(w + part_b + h->ws_max_bytes);
    h->ws_u32_base = reinterpret_cast<unsigned int *>(w + part_b + h->ws_max_bytes + h->ws_min_bytes);
    h->ws.maxv = h->ws_max_base;
    h->ws.minv = h->ws_min_base;
    h->ws.rowany = h->ws_u32_base;
    h->ws.bad = h->ws_u32_base + ny;
    h->ws.gcount = h->ws_u32_base + ny + 3;
    h->ws.gpartials = h->ws.partials + (size_t)nb * OBS_NSUM;
    h->ws.nblocks = obs_grid_blocks(nx, ny);
    h->ws.ngroups = (h->ws.nblocks + OBS_GROUP - 1) / OBS_GROUP;
    h->ws.obs = reinterpret_cast<lbm_obs *>(w + part_b + h->ws_max_bytes + h->ws_min_bytes + h->ws_u32_bytes);
    h->err = reinterpret_cast<unsigned int *>(w + part_b + h->ws_max_bytes + h->ws_min_bytes + h->ws_u32_bytes + obs_b);
    h->s.err = h->err;
    h->s.rng = h->err + 4;     // two counters in the same 256-byte block
    h->qdot = reinterpret_cast<double *>(w + part_b + h->ws_max_bytes + h->ws_min_bytes + h->ws_u32_bytes + obs_b +
                                         err_b);
    if (cudaMemset(h->err, 0, err_b) != cudaSuccess ||
        cudaMemset(h->s.halo, 0, halo_b) != cudaSuccess ||
        cudaMemset(h->ws_max_base, 0x00, h->ws_max_bytes) != cudaSuccess ||
        cudaMemset(h->ws_min_base, 0xFF, h->ws_min_bytes) != cudaSuccess ||
        cudaMemset(h->ws_u32_base, 0x00, h->ws_u32_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->ws_mem);
        cudaFree(h->mem);
        delete h;
        return fail(LBM_ERR_CUDA, "workspace initialisation failed");
    }
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->ws_mem);
        cudaFree(h->mem);
        delete h;
        return fail(LBM_ERR_CUDA, "stream creation failed");
    }
    *out = h;
    return LBM_OK;
}

void lbm_destroy(lbm_handle *h) {
    if (!h) return;
    h->obs_pending = false;      // a requested observation nobody can fetch any more
    cudaStreamSynchronize(h->st);
    drop_graphs(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    cudaFree(h->staging);
    if (h->imp_st) {
        cudaStreamSynchronize(h->imp_st);
        cudaStreamDestroy(h->imp_st);
    }
    for (int j = 0; j < 2; j++) {
        if (h->imp_filled[j]) cudaEventDestroy(h->imp_filled[j]);
        if (h->imp_free[j]) cudaEventDestroy(h->imp_free[j]);
        cudaFree(h->imp_buf[j]);
    }
    cudaFree(h->ws_mem);
    cudaFree(h->mem);
    delete h;
}

int lbm_init_droplet(lbm_handle *h, double R, double xc, double yc, int32_t presolve) {
    if (!h) return fail(LBM_ERR_BADPARAM, "NULL handle");
    if (!(R > 0.0) || presolve < 0 || !std::isfinite(xc) || !std::isfinite(yc))
        return fail(LBM_ERR_BADPARAM, "R must be positive, presolve >= 0, centre finite");
    return finish_init(h, nullptr, R, xc, yc, presolve);
}

int lbm_init_psi(lbm_handle *h, const double *psi, int32_t presolve) {
    if (!h || !psi) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (presolve < 0) return fail(LBM_ERR_BADPARAM, "presolve must be >= 0");
    int rc = ensure_staging(h);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->staging, psi, sizeof(double) * h->P.nx * h->P.ny, cudaMemcpyHostToDevice, h->st));
    return finish_init(h, h->staging, 0.0, 0.0, 0.0, presolve);
}

int lbm_step(lbm_handle *h, int64_t n) {
    if (!h) return fail(LBM_ERR_BADPARAM, "NULL handle");
    if (n < 0) return fail(LBM_ERR_BADPARAM, "n must be >= 0");
    if (!h->inited) return fail(LBM_ERR_STATE, "step before init");
    if (h->diverged) return fail(LBM_ERR_DIVERGED, "instance diverged earlier");
    if (n >= 1 && h->obs_pending) {
        // the first step reads the observed state: it reduces the observables too
        h->obs_pending = false;
        cudaError_t e = do_step(h, h->st, &h->obs_sc);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel with observables");
        if (h->obs_out) {
            lbm_obs *out = h->obs_out;
            h->obs_out = nullptr;
            CK(cudaMemcpyAsync(out, h->ws.obs, sizeof(lbm_obs), cudaMemcpyDeviceToHost, h->st));
        }
        h->step += 1;
        n -= 1;
    }
    // Long runs replay a captured graph of G steps (G even, so both parities
    // return to their starting values and the graph can be reused).
    const int G = 32;
    while (n >= G) {
        cudaGraphExec_t &ex = h->gexec[h->cur][h->lcur];
        if (!ex) {
            const int c0 = h->cur, l0 = h->lcur;
            CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int j = 0; j < G && e == cudaSuccess; j++) e = do_step(h, h->cap);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
            h->cur = c0;
            h->lcur = l0;
            if (e != cudaSuccess) return cuda_fail(e, "graph capture of the step");
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ex = nullptr;
                return cuda_fail(e, "cudaGraphInstantiate");
            }
        }
        CK(cudaGraphLaunch(ex, h->st));
        // G steps flip cur G times and lcur G * k_e times: both even.
        h->step += G;
        n -= G;
    }
    for (int64_t j = 0; j < n; j++) {
        cudaError_t e = do_step(h, h->st);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel");
        h->step += 1;
    }
    return LBM_OK;
}

int lbm_observables_async(lbm_handle *h) {
    if (!h) return fail(LBM_ERR_BADPARAM, "NULL handle");
    if (!h->inited) return fail(LBM_ERR_STATE, "observables before init");
    int rc = run_pending_obs(h);       // an earlier request that no step has taken
    if (rc) return rc;
    // the workspace starts at the identities of its reductions (set at
    // creation) and the finish launch's last block restores them
    Scalars sc;
    sc.step = h->step;
    sc.alpha_l = h->P.alpha_l;
    sc.R0 = h->P.R0;
    cudaError_t e;
    switch (h->P.precision) {
    case LBM_FP64: e = launch_obs_f64(h->s, h->cur, h->lcur, &h->cd, h->sh, h->ws, sc, h->st); break;
    case LBM_FP32: e = launch_obs_f32(h->s, h->cur, h->lcur, &h->cf, h->sh, h->ws, sc, h->st); break;
    default: e = launch_obs_f16s(h->s, h->cur, h->lcur, &h->cf, h->sh, h->ws, sc, h->st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "observables kernels");
    return LBM_OK;
}

int lbm_observables_fetch(lbm_handle *h, lbm_obs *out) {
    if (!h || !out) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (!h->inited) return fail(LBM_ERR_STATE, "observables before init");
    int rc = run_pending_obs(h);
    if (rc) return rc;
    unsigned int err = 0;
    CK(cudaMemcpyAsync(out, h->ws.obs, sizeof(lbm_obs), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&err, h->err, sizeof err, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (err) return fail(LBM_ERR_CUDA, "a kernel reported an error status");
    if (out->status == LBM_ERR_DIVERGED) {
        h->diverged = true;
        return fail(LBM_ERR_DIVERGED, "non-finite psi or H");
    }
    return LBM_OK;
}

int lbm_observables(lbm_handle *h, lbm_obs *out) {
    if (!out) return fail(LBM_ERR_BADPARAM, "NULL argument");
    int rc = lbm_observables_async(h);
    if (rc) return rc;
    return lbm_observables_fetch(h, out);
}

int lbm_observables_to_host(lbm_handle *h, lbm_obs *out) {
    if (!h || !out) return fail(LBM_ERR_BADPARAM, "NULL argument");
    const int rc = lbm_observables_async(h);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out, h->ws.obs, sizeof(lbm_obs), cudaMemcpyDeviceToHost, h->st));
    return LBM_OK;
}

int lbm_observables_deferred(lbm_handle *h, lbm_obs *out) {
    if (!h) return fail(LBM_ERR_BADPARAM, "NULL handle");
    if (!h->inited) return fail(LBM_ERR_STATE, "observables before init");
    int rc = run_pending_obs(h);       // an earlier request that no step has taken
    if (rc) return rc;
    h->obs_pending = true;
    h->obs_sc.step = h->step;
    h->obs_sc.alpha_l = h->P.alpha_l;
    h->obs_sc.R0 = h->P.R0;
    h->obs_out = out;
    return LBM_OK;
}

int lbm_sync(lbm_handle *h) {
    if (!h) return fail(LBM_ERR_BADPARAM, "NULL handle");
    int rc = run_pending_obs(h);
    if (rc) return rc;
    unsigned int err = 0;
    CK(cudaMemcpyAsync(&err, h->err, sizeof err, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (err) return fail(LBM_ERR_CUDA, "a kernel reported an error status");
    return LBM_OK;
}

int lbm_substrate_heat_flux(lbm_handle *h, double *host_out) {
    if (!h || !host_out) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (h->P.ny < 3) return fail(LBM_ERR_BADPARAM, "the substrate heat flux needs ny >= 3");
    if (!h->inited) return fail(LBM_ERR_STATE, "heat flux before init");
    if (int rc_ = run_pending_obs(h)) return rc_;
    cudaError_t e;
    switch (h->P.precision) {
    case LBM_FP64: e = launch_heat_flux_f64(h->s, h->cur, h->lcur, &h->cd, h->sh, h->qdot, h->st); break;
    case LBM_FP32: e = launch_heat_flux_f32(h->s, h->cur, h->lcur, &h->cf, h->sh, h->qdot, h->st); break;
    default: e = launch_heat_flux_f16s(h->s, h->cur, h->lcur, &h->cf, h->sh, h->qdot, h->st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "heat flux kernel");
    CK(cudaMemcpyAsync(host_out, h->qdot, sizeof(double) * h->P.nx, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
}

static int field_planes(int field) {
    if (field == LBM_FIELD_F || field == LBM_FIELD_H || field == LBM_FIELD_G) return 9;
    if (field == LBM_FIELD_L) return 5;
    if (field >= LBM_FIELD_FS_PREV && field <= LBM_FIELD_SIGMA) return 1;
    return 0;
}

int lbm_get_field(lbm_handle *h, int32_t field, double *host_out) {
    if (!h || !host_out) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (int rc_ = run_pending_obs(h)) return rc_;
    const int planes = field_planes(field);
    if (!planes) return fail(LBM_ERR_BADPARAM, "unknown field id");
    if (!h->inited) return fail(LBM_ERR_STATE, "field access before init");
    int rc = ensure_staging(h);
    if (rc) return rc;
    cudaError_t e;
    switch (h->P.precision) {
    case LBM_FP64: e = launch_get_f64(h->s, h->cur, h->lcur, field, &h->cd, h->sh, h->staging, h->st); break;
    case LBM_FP32: e = launch_get_f32(h->s, h->cur, h->lcur, field, &h->cd, h->sh, h->staging, h->st); break;
    default: e = launch_get_f16s(h->s, h->cur, h->lcur, field, &h->cd, h->sh, h->staging, h->st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "field gather kernel");
    CK(cudaMemcpyAsync(host_out, h->staging, sizeof(double) * planes * h->P.nx * h->P.ny,
                       cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
}

int lbm_set_field(lbm_handle *h, int32_t field, const double *host_in) {
    if (!h || !host_in) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (int rc_ = run_pending_obs(h)) return rc_;
    const int planes = field_planes(field);
    if (!planes || (field >= LBM_FIELD_PSI && field <= LBM_FIELD_HTOT))
        return fail(LBM_ERR_BADPARAM, "field id is not writable");
    if (!h->inited) return fail(LBM_ERR_STATE, "field access before init");
    int rc = ensure_staging(h);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->staging, host_in, sizeof(double) * planes * h->P.nx * h->P.ny,
                       cudaMemcpyHostToDevice, h->st));
    const void *c = consts_for(h);
    cudaError_t e;
    switch (h->P.precision) {
    case LBM_FP64: e = launch_set_f64(h->s, h->cur, h->lcur, field, c, h->sh, h->staging, h->st); break;
    case LBM_FP32: e = launch_set_f32(h->s, h->cur, h->lcur, field, c, h->sh, h->staging, h->st); break;
    default: e = launch_set_f16s(h->s, h->cur, h->lcur, field, c, h->sh, h->staging, h->st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "field scatter kernel");
    CK(cudaStreamSynchronize(h->st));
    return LBM_OK;
}

// Snapshot layout: header | f,h,g planes | l planes | aux planes | sigma | lbm_obs
struct SnapHeader {
    char magic[8];
    int64_t step;
    int32_t nx, ny, precision, k_e;
    int64_t body_bytes;
    uint32_t sr_step;      // stochastic-rounding counter of half storage
    int32_t phase;         // layout phases at export: cur | lcur << 1 (the body is natural)
    char pad[16];
};
static_assert(sizeof(SnapHeader) == 64, "snapshot header is 64 bytes");

static void snap_sizes(const lbm_handle *h, size_t &fhg, size_t &l, size_t &aux, size_t &sig) {
    const size_t sb = storage_bytes(h->P.precision), ab = aux_bytes(h->P.precision);
    fhg = l_offset_bytes(h->P.precision, h->s.plane);
    l = (size_t)(NPOP - NFHG) * h->s.plane * sb;
    aux = (size_t)NAUX * h->s.plane * ab;
    sig = (size_t)h->s.plane * ab;
}

size_t lbm_state_bytes(const lbm_handle *h) {
    if (!h) return 0;
    size_t a, b, c, d;
    snap_sizes(h, a, b, c, d);
    return sizeof(SnapHeader) + a + b + c + d + sizeof(lbm_obs);
}

int lbm_export_state(lbm_handle *h, void *host, size_t bytes) {
    if (!h || !host) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (int rc_ = run_pending_obs(h)) return rc_;
    if (bytes != lbm_state_bytes(h)) return fail(LBM_ERR_BADPARAM, "snapshot size mismatch");
    if (!h->inited) return fail(LBM_ERR_STATE, "export before init");
    size_t a, b, c, d;
    snap_sizes(h, a, b, c, d);
    SnapHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, "LBMGB300", 8);
    hd.step = h->step;
    hd.nx = h->P.nx;
    hd.ny = h->P.ny;
    hd.precision = h->P.precision;
    hd.k_e = h->P.k_e;
    hd.body_bytes = (int64_t)(a + b + c + d + sizeof(lbm_obs));
    hd.phase = h->cur | (h->lcur << 1);
    char *o = static_cast<char *>(host);
    std::memcpy(o, &hd, sizeof hd);
    CK(cudaMemcpyAsync(o + offsetof(SnapHeader, sr_step), h->s.rng + h->cur, sizeof(uint32_t),
                       cudaMemcpyDeviceToHost, h->st));
    o += sizeof hd;
    CK(cudaMemcpyAsync(o, h->s.pop, a + b, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(o + a + b, h->s.aux[h->cur], c, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(o + a + b + c, h->s.sigma, d, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(o + a + b + c + d, h->ws.obs, sizeof(lbm_obs), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    // snapshots hold the natural layout whatever the phase of the state
    const int prec = h->P.precision;
    const size_t fb = f_bytes(prec), sb = storage_bytes(prec);
    const long long P = h->s.plane;
    if (h->cur) {
        unswap_planes(o, fb, 9, h->P.nx, h->P.ny, h->s.pitch, P);
        unswap_planes(o + 9 * P * fb, sb, 9, h->P.nx, h->P.ny, h->s.pitch, P);
        unswap_planes(o + 9 * P * fb + 9 * P * sb, sb, 9, h->P.nx, h->P.ny, h->s.pitch, P);
    }
    if (h->lcur) unswap_planes(o + a, sb, 5, h->P.nx, h->P.ny, h->s.pitch, P);
    return LBM_OK;
}

int lbm_import_state(lbm_handle *h, const void *host, size_t bytes) {
    if (!h || !host) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (int rc_ = run_pending_obs(h)) return rc_;
    if (bytes != lbm_state_bytes(h)) return fail(LBM_ERR_BADPARAM, "snapshot size mismatch");
    SnapHeader hd;
    std::memcpy(&hd, host, sizeof hd);
    if (std::memcmp(hd.magic, "LBMGB300", 8) != 0 || hd.nx != h->P.nx || hd.ny != h->P.ny ||
        hd.precision != h->P.precision || hd.k_e != h->P.k_e)
        return fail(LBM_ERR_BADPARAM, "snapshot does not match this handle");
    if (!h->imp_st) {
        // buffers, events and the copy stream, all or none
        bool ok = cudaMalloc(&h->imp_buf[0], bytes) == cudaSuccess && cudaMalloc(&h->imp_buf[1], bytes) == cudaSuccess;
        const bool oom = !ok;
        for (int j = 0; j < 2 && ok; j++)
            ok = cudaEventCreateWithFlags(&h->imp_filled[j], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->imp_free[j], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&h->imp_st, cudaStreamNonBlocking) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (int j = 0; j < 2; j++) {
                if (h->imp_filled[j]) cudaEventDestroy(h->imp_filled[j]);
                if (h->imp_free[j]) cudaEventDestroy(h->imp_free[j]);
                cudaFree(h->imp_buf[j]);
                h->imp_filled[j] = h->imp_free[j] = nullptr;
                h->imp_buf[j] = nullptr;
            }
            h->imp_st = nullptr;
            return oom ? fail(LBM_ERR_OOM, "device allocation of the import buffers failed")
                       : fail(LBM_ERR_CUDA, "events or stream of the import path could not be created");
        }
    }
    // the whole snapshot to device buffer j on the import stream, once the
    // handle's stream has unpacked what buffer j held before (an event never
    // recorded is no wait); then the handle's stream unpacks it
    const int j = h->imp_next;
    h->imp_next ^= 1;
    const char *dev = static_cast<const char *>(h->imp_buf[j]);
    CK(cudaStreamWaitEvent(h->imp_st, h->imp_free[j], 0));
    CK(cudaMemcpyAsync(h->imp_buf[j], host, bytes, cudaMemcpyHostToDevice, h->imp_st));
    CK(cudaEventRecord(h->imp_filled[j], h->imp_st));
    CK(cudaStreamWaitEvent(h->st, h->imp_filled[j], 0));
    size_t a, b, c, d;
    snap_sizes(h, a, b, c, d);
    const char *o = dev + sizeof hd;
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    // the body holds the natural layout; the state resumes in the layout
    // phases it was exported at, so the same step kernels follow (single
    // precision rounds each phase's kernel in its own way)
    if (hd.phase < 0 || hd.phase > 3) return fail(LBM_ERR_BADPARAM, "snapshot layout phase out of range");
    h->cur = hd.phase & 1;
    h->lcur = (hd.phase >> 1) & 1;
    if (hd.phase == 0) {
        CK(cudaMemcpyAsync(h->s.pop, o, a + b, dd, h->st));
    } else {
        cudaError_t e;
        switch (h->P.precision) {
        case LBM_FP64: e = launch_place_f64(h->s, h->cur, h->lcur, o, h->st); break;
        case LBM_FP32: e = launch_place_f32(h->s, h->cur, h->lcur, o, h->st); break;
        default: e = launch_place_f16s(h->s, h->cur, h->lcur, o, h->st); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "snapshot placement kernel");
    }
    CK(cudaMemcpyAsync(h->s.aux[h->cur], o + a + b, c, dd, h->st));
    CK(cudaMemcpyAsync(h->s.sigma, o + a + b + c, d, dd, h->st));
    CK(cudaMemcpyAsync(h->ws.obs, o + a + b + c + d, sizeof(lbm_obs), dd, h->st));
    CK(cudaMemcpyAsync(h->s.rng + h->cur, dev + offsetof(SnapHeader, sr_step), sizeof(uint32_t), dd, h->st));
    CK(cudaEventRecord(h->imp_free[j], h->st));
    h->step = hd.step;
    h->inited = true;
    h->diverged = false;
    return LBM_OK;
}

int lbm_presolve(lbm_handle *h, double tol, int32_t max_sweeps, int32_t *sweeps, double *residual) {
    if (!h) return fail(LBM_ERR_BADPARAM, "NULL handle");
    if (!(tol > 0.0) || max_sweeps < 1) return fail(LBM_ERR_BADPARAM, "tol must be > 0 and max_sweeps >= 1");
    if (!h->inited) return fail(LBM_ERR_STATE, "pre-solve before init");
    if (int rc_ = run_pending_obs(h)) return rc_;
    const double dphi = std::fabs(h->cd.phi_top - h->cd.phi_bot);
    const double scale = dphi > 0.0 ? dphi : 1.0;
    // the observables workspace's spare maximum slot holds the change
    unsigned long long *d = h->ws.maxv + 1;
    const int chunk = 64;        // sweeps between two measurements
    int done = 0;
    double res = HUGE_VAL;
    // phi before the last sweep of each chunk goes to the spare auxiliary
    // copy (the next step overwrites it without reading it)
    void *snap = h->s.aux[h->cur ^ 1];
    while (done < max_sweeps) {
        const int n = std::min(chunk, max_sweeps - done);
        for (int j = 0; j < n; j++) {
            cudaError_t e = cudaSuccess;
            if (j == n - 1) {
                switch (h->P.precision) {
                case LBM_FP64: e = launch_phi_snap_f64(h->s, h->lcur, &h->cd, h->sh, snap, h->st); break;
                case LBM_FP32: e = launch_phi_snap_f32(h->s, h->lcur, &h->cd, h->sh, snap, h->st); break;
                default: e = launch_phi_snap_f16s(h->s, h->lcur, &h->cd, h->sh, snap, h->st); break;
                }
                if (e != cudaSuccess) return cuda_fail(e, "pre-solve snapshot");
            }
            e = do_sweep(h, h->st);
            if (e != cudaSuccess) return cuda_fail(e, "pre-solve sweep");
        }
        done += n;
        // change of phi over the last sweep
        CK(cudaMemsetAsync(d, 0, sizeof *d, h->st));
        cudaError_t e;
        switch (h->P.precision) {
        case LBM_FP64: e = launch_phi_change_f64(h->s, h->lcur, &h->cd, h->sh, snap, d, h->st); break;
        case LBM_FP32: e = launch_phi_change_f32(h->s, h->lcur, &h->cd, h->sh, snap, d, h->st); break;
        default: e = launch_phi_change_f16s(h->s, h->lcur, &h->cd, h->sh, snap, d, h->st); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "pre-solve residual");
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, d, sizeof bits, cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemsetAsync(d, 0, sizeof *d, h->st));      // the slot's identity again
        CK(cudaStreamSynchronize(h->st));
        double change;
        std::memcpy(&change, &bits, sizeof change);
        res = change / scale;
        if (res < tol) break;
        if (!std::isfinite(res)) {
            if (sweeps) *sweeps = done;
            if (residual) *residual = res;
            return fail(LBM_ERR_DIVERGED, "non-finite potential in the pre-solve");
        }
    }
    if (sweeps) *sweeps = done;
    if (residual) *residual = res;
    if (res < tol) return LBM_OK;
    return fail(LBM_WARN_NOT_CONVERGED, "pre-solve stopped at max_sweeps above the tolerance");
}

int64_t lbm_step_count(const lbm_handle *h) { return h ? h->step : -1; }

}  // extern "C"

namespace lbm {
// half_round.cu (built with the half-storage step's flags)
cudaError_t launch_round_half_sr(const float *v, const uint32_t *r, uint16_t *out, long long n, cudaStream_t st);
}

extern "C" {

int lbm_round_half_sr(const float *v, const uint32_t *r, uint16_t *out, int64_t n, void *stream) {
    if (n < 0) return fail(LBM_ERR_BADPARAM, "negative count");
    if (n == 0) return LBM_OK;
    if (!v || !r || !out) return fail(LBM_ERR_BADPARAM, "NULL argument");
    if (reinterpret_cast<uintptr_t>(v) % 4 || reinterpret_cast<uintptr_t>(r) % 4 ||
        reinterpret_cast<uintptr_t>(out) % 2)
        return fail(LBM_ERR_BADPARAM, "misaligned pointer");
    CK(launch_round_half_sr(v, r, out, (long long)n, static_cast<cudaStream_t>(stream)));
    return LBM_OK;
}

size_t lbm_device_bytes(const lbm_handle *h) {
    if (!h) return 0;
    size_t n = h->mem_bytes + h->ws_mem_bytes;
    if (h->staging) n += (size_t)9 * h->P.nx * h->P.ny * sizeof(double);
    if (h->imp_buf[0]) n += 2 * lbm_state_bytes(h);
    return n;
}

int lbm_configure(lbm_handle *h, int32_t variant, int32_t tile_rows) {
    if (!h) return fail(LBM_ERR_BADPARAM, "NULL handle");
    if (int rc_ = run_pending_obs(h)) return rc_;
    if (variant != LBM_STEP_DIRECT) return fail(LBM_ERR_BADPARAM, "unknown variant");
    if (tile_rows != 4 && tile_rows != 8 && tile_rows != 16) return fail(LBM_ERR_BADPARAM, "tile_rows must be 4, 8 or 16");
    CK(cudaStreamSynchronize(h->st));
    h->tile_rows = tile_rows;
    h->variant = variant;
    drop_graphs(h);
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------

static cudaError_t list_steps(const lbm_batch *b, const WorkList &L, int64_t n, int &flips, int &lflips,
                              cudaStream_t st) {
    for (int64_t j = 0; j < n; j++) {
        const int fc = flips & 1, fl = lflips & 1;
        cudaError_t e;
        switch (b->precision) {
        case LBM_FP64:
            e = launch_batch_step_f64(L.items_dev, L.consts_dev, L.tile_item_dev, L.total_tiles, b->tile_rows, L.grid,
                                       fc, fl, st);
            break;
        case LBM_FP32:
            e = launch_batch_step_f32(L.items_dev, L.consts_dev, L.tile_item_dev, L.total_tiles, b->tile_rows, L.grid,
                                       fc, fl, st);
            break;
        default:
            e = launch_batch_step_f16s(L.items_dev, L.consts_dev, L.tile_item_dev, L.total_tiles, b->tile_rows, L.grid,
                                       fc, fl, st);
            break;
        }
        if (e != cudaSuccess) return e;
        flips++;
        lflips++;
        for (int sw = 1; sw < b->k_e; sw++) {
            const int fl2 = lflips & 1, fc2 = flips & 1;
            const uint32_t sys = 3u + (uint32_t)sw;   // as the single-instance sweeps
            switch (b->precision) {
            case LBM_FP64:
                e = launch_batch_sweep_f64(L.items_dev, L.consts_dev, L.n, L.total_sweep_tiles, L.sweep_grid, fl2, fc2,
                                           sys, st);
                break;
            case LBM_FP32:
                e = launch_batch_sweep_f32(L.items_dev, L.consts_dev, L.n, L.total_sweep_tiles, L.sweep_grid, fl2, fc2,
                                           sys, st);
                break;
            default:
                e = launch_batch_sweep_f16s(L.items_dev, L.consts_dev, L.n, L.total_sweep_tiles, L.sweep_grid, fl2,
                                            fc2, sys, st);
                break;
            }
            if (e != cudaSuccess) return e;
            lflips++;
        }
    }
    return cudaSuccess;
}

static void free_list(WorkList &L) {
    for (int a = 0; a < 2; a++)
        for (int c = 0; c < 2; c++)
            if (L.gexec[a][c]) {
                cudaGraphExecDestroy(L.gexec[a][c]);
                L.gexec[a][c] = nullptr;
            }
    cudaFree(L.items_dev);
    cudaFree(L.consts_dev);
    cudaFree(L.tile_item_dev);
    L.items_dev = nullptr;
    L.consts_dev = nullptr;
    L.tile_item_dev = nullptr;
}

// Device bytes a member's step touches: the populations (one copy, in
// place), both auxiliary copies, sigma and the halo records.
static size_t member_state_bytes(const lbm_handle *h) {
    const int prec = h->P.precision;
    const size_t ab = aux_bytes(prec);
    return (size_t)h->s.plane * (pop_cell_bytes(prec) + 2 * NAUX * ab + ab + halo_rec_bytes(prec));
}

static int build_list(lbm_batch *b, const std::vector<int> &idx, int tile_rows, int sms, WorkList &L) {
    free_list(L);
    std::vector<BatchItem> items(idx.size());
    const size_t csz = b->precision == LBM_FP64 ? sizeof(Consts<double>) : sizeof(Consts<float>);
    std::vector<char> cs(csz * idx.size());
    int tiles = 0, sweeps = 0;
    for (size_t j = 0; j < idx.size(); j++) {
        lbm_handle *h = b->m[idx[j]];
        BatchItem &it = items[j];
        it.s = h->s;
        it.cur = h->cur;
        it.lcur = h->lcur;
        it.write_sigma = h->P.k_e > 1 ? 1 : 0;
        it.tiles_x = (h->P.nx + 31) / 32;
        it.tiles_y = (h->P.ny + tile_rows - 1) / tile_rows;
        it.tile_begin = tiles;
        tiles += it.tiles_x * it.tiles_y;
        it.sweep_tiles_x = it.tiles_x;
        it.sweep_begin = sweeps;
        sweeps += it.tiles_x * ((h->P.ny + 7) / 8);
        it.sh = h->sh;
        std::memcpy(cs.data() + csz * j, consts_for(h), csz);
    }
    L.n = (int)idx.size();
    L.total_tiles = tiles;
    L.total_sweep_tiles = sweeps;
    std::vector<int> tile_item(tiles);
    for (size_t j = 0; j < items.size(); j++)
        for (int t = 0; t < items[j].tiles_x * items[j].tiles_y; t++) tile_item[items[j].tile_begin + t] = (int)j;
    // persistent grid = the blocks the device holds at once
    const int per_sm = b->precision == LBM_FP64 ? batch_blocks_per_sm_f64(tile_rows)
                     : b->precision == LBM_FP32 ? batch_blocks_per_sm_f32(tile_rows)
                                                : batch_blocks_per_sm_f16s(tile_rows);
    if (per_sm < 1) return fail(LBM_ERR_CUDA, "occupancy query of the batched step failed");
    L.grid = std::min(tiles, sms * per_sm);
    L.sweep_grid = std::min(sweeps, sms * 8);
    CK(cudaMalloc(&L.items_dev, items.size() * sizeof(BatchItem)));
    CK(cudaMalloc(&L.consts_dev, cs.size()));
    CK(cudaMalloc(&L.tile_item_dev, sizeof(int) * (size_t)std::max(tiles, 1)));
    CK(cudaMemcpyAsync(L.items_dev, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, b->st));
    CK(cudaMemcpyAsync(L.consts_dev, cs.data(), cs.size(), cudaMemcpyHostToDevice, b->st));
    CK(cudaMemcpyAsync(L.tile_item_dev, tile_item.data(), sizeof(int) * tile_item.size(), cudaMemcpyHostToDevice,
                       b->st));
    // the host vectors go out of scope on return: finish the copies first
    CK(cudaStreamSynchronize(b->st));
    return LBM_OK;
}

// Build the all-member list and the L2-sized groups (consecutive members
// whose combined state stays within half of the L2 cache).
static int batch_build(lbm_batch *b, int tile_rows) {
    int dev = 0, sms = 0, l2 = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    b->tile_rows = tile_rows;
    std::vector<int> all(b->m.size());
    for (size_t i = 0; i < all.size(); i++) all[i] = (int)i;
    int rc = build_list(b, all, tile_rows, sms, b->all);
    if (rc) return rc;
    for (WorkList &g : b->groups) free_list(g);
    b->groups.clear();
    const size_t budget = (size_t)l2 / 2;
    std::vector<int> cur;
    size_t used = 0;
    for (size_t i = 0; i <= b->m.size(); i++) {
        const bool end = (i == b->m.size());
        const size_t need = end ? 0 : member_state_bytes(b->m[i]);
        if (!cur.empty() && (end || used + need > budget)) {
            b->groups.emplace_back();
            if ((rc = build_list(b, cur, tile_rows, sms, b->groups.back()))) return rc;
            cur.clear();
            used = 0;
        }
        if (!end) {
            cur.push_back((int)i);
            used += need;
        }
    }
    CK(cudaStreamSynchronize(b->st));
    b->cur0.resize(b->m.size());
    b->lcur0.resize(b->m.size());
    for (size_t i = 0; i < b->m.size(); i++) {
        b->cur0[i] = b->m[i]->cur;
        b->lcur0[i] = b->m[i]->lcur;
    }
    b->flips = 0;
    b->lflips = 0;
    return LBM_OK;
}

// n steps of one list starting at parities (flips, lflips); long runs replay
// a captured graph of G steps (G even: both parities return to the start).
static int run_list(lbm_batch *b, WorkList &L, int64_t n, int flips, int lflips) {
    const int G = 32;
    while (n >= G) {
        cudaGraphExec_t &ex = L.gexec[flips & 1][lflips & 1];
        if (!ex) {
            int f = flips, lf = lflips;
            CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = list_steps(b, L, G, f, lf, b->cap);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
            if (e != cudaSuccess) return cuda_fail(e, "graph capture of the batch step");
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ex = nullptr;
                return cuda_fail(e, "cudaGraphInstantiate");
            }
        }
        CK(cudaGraphLaunch(ex, b->st));
        flips += G;
        lflips += G * b->k_e;
        n -= G;
    }
    cudaError_t e = list_steps(b, L, n, flips, lflips, b->st);
    if (e != cudaSuccess) return cuda_fail(e, "batch step");
    return LBM_OK;
}

int lbm_batch_create(lbm_handle *const *members, int32_t n, void *stream, int32_t tile_rows, lbm_batch **out) {
    if (!members || !out || n < 1) return fail(LBM_ERR_BADPARAM, "need at least one member");
    *out = nullptr;
    if (tile_rows != 0 && tile_rows != 4 && tile_rows != 8 && tile_rows != 16)
        return fail(LBM_ERR_BADPARAM, "tile_rows must be 0, 4, 8 or 16");
    for (int i = 0; i < n; i++) {
        if (!members[i]) return fail(LBM_ERR_BADPARAM, "NULL member");
        if (!members[i]->inited) return fail(LBM_ERR_STATE, "member not initialised");
        if (members[i]->P.precision != members[0]->P.precision)
            return fail(LBM_ERR_BADPARAM, "members must share the precision");
        if (members[i]->P.k_e != members[0]->P.k_e) return fail(LBM_ERR_BADPARAM, "members must share k_e");
        if (members[i]->diverged) return fail(LBM_ERR_DIVERGED, "member diverged earlier");
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return fail(LBM_ERR_OOM, "host allocation failed");
    b->m.assign(members, members + n);
    b->precision = members[0]->P.precision;
    b->k_e = members[0]->P.k_e;
    b->st = static_cast<cudaStream_t>(stream);
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(LBM_ERR_CUDA, "stream creation failed");
    }
    int rc = LBM_OK;
    if (tile_rows == 0) {
        // Autotune: time each tile height on the members' own data.  The
        // steps stream in place, so the trials advance the members' state
        // (six steps per height, an even number: the layout phases return)
        // and overwrite both auxiliary copies; the state they started from
        // (populations, auxiliary copies, sigma, counters) is saved first
        // and put back after.
        std::vector<size_t> pop_sz(n), sig_sz(n), aux_sz(n);
        size_t total = 0;
        for (int i = 0; i < n; i++) {
            const lbm_handle *h = members[i];
            pop_sz[i] = (size_t)h->s.plane * pop_cell_bytes(h->P.precision);
            sig_sz[i] = (size_t)h->s.plane * aux_bytes(h->P.precision);
            aux_sz[i] = (size_t)NAUX * h->s.plane * aux_bytes(h->P.precision);
            total += round_up(pop_sz[i], 256) + round_up(sig_sz[i], 256) + 2 * round_up(aux_sz[i], 256) + 256;
        }
        char *saved = nullptr;
        if (cudaMalloc(&saved, total) != cudaSuccess) {
            cudaGetLastError();
            lbm_batch_destroy(b);
            return fail(LBM_ERR_OOM, "device allocation of the autotuner's saved state failed");
        }
        auto copy_members = [&](bool save) -> cudaError_t {
            size_t off = 0;
            for (int i = 0; i < n; i++) {
                const lbm_handle *h = members[i];
                char *a = saved + off, *bb = a + round_up(pop_sz[i], 256), *x0 = bb + round_up(sig_sz[i], 256);
                char *x1 = x0 + round_up(aux_sz[i], 256), *cnt = x1 + round_up(aux_sz[i], 256);
                off += round_up(pop_sz[i], 256) + round_up(sig_sz[i], 256) + 2 * round_up(aux_sz[i], 256) + 256;
                const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
                cudaError_t e = cudaMemcpyAsync(save ? a : h->s.pop, save ? h->s.pop : a, pop_sz[i], dd, b->st);
                if (e == cudaSuccess) e = cudaMemcpyAsync(save ? bb : h->s.sigma, save ? h->s.sigma : bb, sig_sz[i], dd, b->st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(save ? x0 : h->s.aux[0], save ? h->s.aux[0] : x0, aux_sz[i], dd, b->st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(save ? x1 : h->s.aux[1], save ? h->s.aux[1] : x1, aux_sz[i], dd, b->st);
                // the status word and rounding counters
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(save ? static_cast<void *>(cnt) : static_cast<void *>(h->err),
                                        save ? static_cast<const void *>(h->err) : static_cast<const void *>(cnt), 64, dd,
                                        b->st);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        };
        float best = 1e30f;
        int best_rows = 8;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaError_t es = copy_members(true);
        if (es != cudaSuccess) rc = cuda_fail(es, "autotune save");
        for (int rows : {4, 8, 16}) {
            if (rc) break;
            if ((rc = batch_build(b, rows))) break;
            const int k_e = b->k_e;
            b->k_e = 1;
            int f = 0, lf = 0;
            cudaError_t e = list_steps(b, b->all, 1, f, lf, b->st);       // warm-up
            cudaEventRecord(e0, b->st);
            for (int r = 0; r < 5 && e == cudaSuccess; r++) e = list_steps(b, b->all, 1, f, lf, b->st);
            cudaEventRecord(e1, b->st);
            b->k_e = k_e;
            if (e != cudaSuccess) { rc = cuda_fail(e, "autotune launch"); break; }
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(LBM_ERR_CUDA, "autotune sync"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; best_rows = rows; }
        }
        es = copy_members(false);
        if (es != cudaSuccess && !rc) rc = cuda_fail(es, "autotune restore");
        if (cudaStreamSynchronize(b->st) != cudaSuccess && !rc) rc = fail(LBM_ERR_CUDA, "autotune restore sync");
        cudaFree(saved);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tile_rows = best_rows;
    }
    if (!rc) rc = batch_build(b, tile_rows);
    if (rc) {
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int64_t n) {
    if (!b) return fail(LBM_ERR_BADPARAM, "NULL batch");
    if (n < 0) return fail(LBM_ERR_BADPARAM, "n must be >= 0");
    for (lbm_handle *h : b->m)
        if (h->diverged) return fail(LBM_ERR_DIVERGED, "a member diverged earlier");
    // a member's deferred observation runs alone, before the batch overwrites
    // its state (on the member's stream: wait for it if that is another one)
    for (lbm_handle *h : b->m) {
        if (!h->obs_pending) continue;
        if (int rc = run_pending_obs(h)) return rc;
        if (h->st != b->st) CK(cudaStreamSynchronize(h->st));
    }
    // A member stepped alone since the list was built has other parities:
    // rebuild the list from the members' current state.
    for (size_t i = 0; i < b->m.size(); i++) {
        if (b->m[i]->cur != (b->cur0[i] ^ (b->flips & 1)) || b->m[i]->lcur != (b->lcur0[i] ^ (b->lflips & 1))) {
            int rc = batch_build(b, b->tile_rows);
            if (rc) return rc;
            break;
        }
    }
    const int64_t total = n;
    // Members are independent: for longer runs each L2-sized group advances
    // all n steps while its state is resident, instead of streaming every
    // member's state through HBM on every step.
    if (n >= 8 && b->groups.size() > 1) {
        for (WorkList &g : b->groups) {
            int rc = run_list(b, g, n, b->flips, b->lflips);
            if (rc) return rc;
        }
    } else {
        int rc = run_list(b, b->all, n, b->flips, b->lflips);
        if (rc) return rc;
    }
    b->flips += (int)(n & 1);
    b->lflips += (int)((n * b->k_e) & 1);
    for (lbm_handle *h : b->m) {
        h->cur ^= (int)(total & 1);
        h->lcur ^= (int)((total * h->P.k_e) & 1);
        h->step += total;
    }
    return LBM_OK;
}

int32_t lbm_batch_tile_rows(const lbm_batch *b) { return b ? b->tile_rows : 0; }

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->st);
    free_list(b->all);
    for (WorkList &g : b->groups) free_list(g);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"
