// Library-internal declarations shared by the translation units of the GPU
// library (host API, and one kernel unit per storage precision).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/lbm.h"

namespace lbm {

// Number of stored planes.
constexpr int NPOP = 32;      // f 9, h 9, g 9, l 5
constexpr int NFHG = 27;      // planes of f, h, g (l follows at plane 27)
constexpr int NAUX = 7;       // fs, mdot, Q, psi*ux, psi*uy, p, S of the previous step
enum { AUX_FS = 0, AUX_MDOT = 1, AUX_Q = 2, AUX_PUX = 3, AUX_PUY = 4, AUX_P = 5, AUX_S = 6 };

// Lattice constants in the arithmetic type T, derived on the host once
// (Secs. 2-3; phase index 0 solid, 1 liquid, 2 gas).
template <typename T>
struct Consts {
    T rho[3], mu[3], kth[3], cp[3], eps[3], sig[3];
    T L, Cref, kappa, beta, tau_f, phi_bot, phi_top, wet, T_m, W;
    T one_m_rsl;     // 1 - rho_s / rho_l
    T Cref_Tw;       // C_p,ref T_w (anti-bounce-back value of g at the cold wall)
    T T_init;
    // reciprocals of the single-precision collision form
    T om_f, pre_f, four_over_W, three_over_Cref;
};

// Reference state subtracted before half-precision storage (weight-shifted
// populations); unused by the FP32/FP64 paths.
struct Shift {
    float f_ref;     // f_i stored as f_i - w_i f_ref
    float g_ref;     // g_i stored as g_i - w_i g_ref (i > 0), g_0 - g0_ref
    float g0_ref;
    float h_scale;   // h_i stored as h_i * h_scale
    float l_scale;   // l_i - w_i phi_lin(y) stored times l_scale
    float f_scale;
    float g_scale;
};

// Views of one instance's device state (element pointers).
struct DevState {
    void *pop;             // one copy of NPOP planes, streamed in place (AA pattern)
    void *aux[2];          // two copies of NAUX planes
    void *sigma;           // one plane
    void *halo;            // one record (psi, f_s, phi) per cell, arithmetic type
    unsigned int *err;     // device status word (sticky error bits)
    unsigned int *rng;     // [2] stochastic-rounding step counters of half storage (or null)
    int nx, ny, pitch;     // pitch: elements per row (multiple of 32)
    long long plane;       // elements per plane (pitch * ny)
};

// Workspace of the observables reduction.
constexpr int OBS_NSUM = 7;          // block sums: psi, H, f_s, q_v, liquid, liquid speed, Qdot
constexpr int OBS_GROUP = 32;        // blocks per first-level group of the final reduction
struct ObsScratch {
    double *partials;               // [nblocks][OBS_NSUM]
    double *gpartials;              // [ngroups][OBS_NSUM]: sums of each group of OBS_GROUP blocks
    unsigned int *gcount;           // [ngroups]: kept at zero (the finish launch has one block per group)
    unsigned long long *maxv;       // [2 + ny]: height, (unused), rightmost crossing of row y
    unsigned long long *minv;       // [1 + ny]: front crossing, leftmost crossing of row y
    unsigned int *rowany;           // [ny]: bit0 liquid, bit1 left crossing, bit2 right crossing
    unsigned int *bad;              // [3]: non-finite seen, centre-column bottom cell frozen,
                                    //      finish blocks done (the last one writes the observables)
    lbm_obs *obs;                   // device-side result (keeps t_fre)
    int nblocks, ngroups;
};

struct Scalars {           // per-call scalars of the observables reduction
    int64_t step;
    double alpha_l, R0;
};

// Precision-specific launchers (one definition per kernel unit).  All
// return cudaSuccess or the launch error; they enqueue on `st`.
#define LBM_DECLARE_LAUNCHERS(SUFFIX)                                                         \
    cudaError_t launch_step_##SUFFIX(const DevState &s, int cur, int lcur, int write_sigma,    \
                                     const void *consts, const Shift &sh, int tile_rows,       \
                                     int variant, cudaStream_t st);                            \
    cudaError_t launch_sweep_##SUFFIX(const DevState &s, int lcur, int cur, uint32_t sr_sys,   \
                                      const void *consts, const Shift &sh, cudaStream_t st);  \
    cudaError_t launch_init_##SUFFIX(const DevState &s, const double *psi_dev, double R,       \
                                     double xc, double yc, const void *consts,                 \
                                     const Shift &sh, cudaStream_t st);                        \
    cudaError_t launch_obs_##SUFFIX(const DevState &s, int cur, int lcur,                      \
                                    const void *consts /* Consts of the step's type */,       \
                                    const Shift &sh, const ObsScratch &ws, const Scalars &sc,  \
                                    cudaStream_t st);                                          \
    cudaError_t launch_step_obs_##SUFFIX(const DevState &s, int cur, int lcur, int write_sigma, \
                                         const void *consts, const Shift &sh, int tile_rows,   \
                                         const ObsScratch &ws, const Scalars &sc,              \
                                         cudaStream_t st);                                      \
    cudaError_t launch_heat_flux_##SUFFIX(const DevState &s, int cur, int lcur,                \
                                          const void *consts /* Consts of the step's type */, \
                                          const Shift &sh, double *out, cudaStream_t st);      \
    cudaError_t launch_get_##SUFFIX(const DevState &s, int cur, int lcur, int field,           \
                                    const void *consts, const Shift &sh, double *out,          \
                                    cudaStream_t st);                                          \
    cudaError_t launch_phi_snap_##SUFFIX(const DevState &s, int lcur,                          \
                                         const void *consts /* Consts<double> */,             \
                                         const Shift &sh, void *snap, cudaStream_t st);        \
    cudaError_t launch_phi_change_##SUFFIX(const DevState &s, int lcur,                        \
                                           const void *consts /* Consts<double> */,           \
                                           const Shift &sh, const void *snap,                  \
                                           unsigned long long *out, cudaStream_t st);          \
    cudaError_t launch_place_##SUFFIX(const DevState &s, int cur, int lcur, const void *src,   \
                                      cudaStream_t st);                                        \
    cudaError_t launch_set_##SUFFIX(const DevState &s, int cur, int lcur, int field,           \
                                    const void *consts, const Shift &sh, const double *in,     \
                                    cudaStream_t st);

LBM_DECLARE_LAUNCHERS(f64)
LBM_DECLARE_LAUNCHERS(f32)
LBM_DECLARE_LAUNCHERS(f16s)

int obs_blocks(int nx, int ny);   // grid size of the observables kernel
void set_last_error(const std::string &msg);
int derive_for_noalloc(const lbm_params *p, Consts<double> *cd, Consts<float> *cf, Shift *sh, const char **why);

// Batched stepping: one launch over a work list of (instance, tile) pairs.
// cur/lcur are the member's parities when the list was built; launches
// pass the number of flips since then (mod 2).
struct BatchItem {
    DevState s;
    int cur, lcur, write_sigma;
    int tiles_x, tiles_y, tile_begin;   // step tiles of this member: [tile_begin, + tiles_x * tiles_y)
    int sweep_tiles_x, sweep_begin;     // 32 x 8 sweep tiles: [sweep_begin, + sweep_tiles_x * ceil(ny/8))
    Shift sh;
};
#define LBM_DECLARE_BATCH(SUFFIX)                                                                  \
    int batch_blocks_per_sm_##SUFFIX(int tile_rows);   /* resident blocks of the batched step */   \
    cudaError_t launch_batch_step_##SUFFIX(const BatchItem *items_dev, const void *consts_dev,     \
                                           const int *tile_item_dev, int total_tiles,              \
                                           int tile_rows, int grid, int flip_cur, int flip_l,      \
                                           cudaStream_t st);                                       \
    cudaError_t launch_batch_sweep_##SUFFIX(const BatchItem *items_dev, const void *consts_dev,    \
                                            int n_items, int total_tiles, int grid, int flip_l,    \
                                            int flip_cur, uint32_t sr_sys, cudaStream_t st);
LBM_DECLARE_BATCH(f64)
LBM_DECLARE_BATCH(f32)
LBM_DECLARE_BATCH(f16s)

}  // namespace lbm
