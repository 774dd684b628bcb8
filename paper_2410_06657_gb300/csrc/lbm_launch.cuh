// Host launchers of the kernels of one precision: LBM_DEFINE_LAUNCHERS(SUFFIX,
// S, T, A) defines the launch_*_SUFFIX functions declared in lbm_internal.h.
#pragma once

#include <utility>

#include "lbm_kernels.cuh"
#include "lbm_observe.cuh"

namespace lbm {

// Launch with programmatic stream serialisation: the kernel may start while
// the one before it in the stream drains, and synchronises with it through
// grid_dep_wait() (lbm_kernels.cuh) before it reads what that kernel wrote.
template <typename... P, typename... Args>
cudaError_t launch_dependent(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Resident blocks per SM of the batched step: the persistent grid is exactly
// the device's resident capacity, so every block starts at once and the
// round-robin tile share is even.
template <typename S, typename T, typename A, int BY>
int batch_blocks_per_sm_by() {
    int n = 0;
    static std::atomic<unsigned long long> ready{0ull};
    if (allow_dynamic_smem(k_batch_step<S, T, A, BY>, stash_bytes<T, BY>(), ready) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<S, T, A, BY>, 32 * BY,
                                                      stash_bytes<T, BY>()) != cudaSuccess)
        return 0;
    return n;
}

template <typename S, typename T, typename A>
int batch_blocks_per_sm_t(int tile_rows) {
    switch (tile_rows) {
    case 4: return batch_blocks_per_sm_by<S, T, A, 4>();
    case 8: return batch_blocks_per_sm_by<S, T, A, 8>();
    case 16: return batch_blocks_per_sm_by<S, T, A, 16>();
    default: return 0;
    }
}

template <typename S, typename T, typename A, int BY>
cudaError_t launch_batch_step_by(const BatchItem *items, const Consts<T> *c, const int *tile_item, int total_tiles,
                                 int grid, int flip_cur, int flip_l, cudaStream_t st) {
    static std::atomic<unsigned long long> ready{0ull};
    cudaError_t e = allow_dynamic_smem(k_batch_step<S, T, A, BY>, stash_bytes<T, BY>(), ready);
    if (e != cudaSuccess) return e;
    const int hgrid = total_tiles < 4 * grid ? total_tiles : 4 * grid;
    e = launch_dependent(k_batch_halo<S, T, A, BY>, dim3(hgrid), dim3(HALO_THREADS), 0, st, items, c, tile_item,
                         total_tiles, flip_cur, flip_l);
    if (e != cudaSuccess) return e;
    return launch_dependent(k_batch_step<S, T, A, BY>, dim3(grid), dim3(32, BY), stash_bytes<T, BY>(), st, items, c,
                            tile_item, total_tiles, flip_cur, flip_l);
}

template <typename S, typename T, typename A>
cudaError_t launch_batch_step_t(const BatchItem *items, const void *consts, const int *tile_item, int total_tiles,
                                int tile_rows, int grid, int flip_cur, int flip_l, cudaStream_t st) {
    const Consts<T> *c = reinterpret_cast<const Consts<T> *>(consts);
    switch (tile_rows) {
    case 4: return launch_batch_step_by<S, T, A, 4>(items, c, tile_item, total_tiles, grid, flip_cur, flip_l, st);
    case 8: return launch_batch_step_by<S, T, A, 8>(items, c, tile_item, total_tiles, grid, flip_cur, flip_l, st);
    case 16: return launch_batch_step_by<S, T, A, 16>(items, c, tile_item, total_tiles, grid, flip_cur, flip_l, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename S, typename T, typename A>
cudaError_t launch_batch_sweep_t(const BatchItem *items, const void *consts, int n_items, int total_tiles, int grid,
                                 int flip_l, int flip_cur, uint32_t sr_sys, cudaStream_t st) {
    const Consts<T> *c = reinterpret_cast<const Consts<T> *>(consts);
    k_batch_sweep<S, T, A><<<grid, dim3(32, 8), 0, st>>>(items, c, n_items, total_tiles, flip_l, flip_cur, sr_sys);
    return cudaGetLastError();
}

// The halo records of a step (first launch of every step).
template <typename S, typename T, typename A, int BY, int PH>
cudaError_t launch_halo_ph(const StepIO<S, T, A> &io, const Consts<T> &c, const Shift &sh, dim3 grid,
                           cudaStream_t st) {
    return launch_dependent(k_halo<S, T, A, BY, PH>, grid, dim3(HALO_THREADS), 0, st, io, c, sh);
}

// The fused step of one instance, tile height BY, from layout phase PH:
// its halo records, then the step itself.
template <typename S, typename T, typename A, int BY, int PH>
cudaError_t launch_step_ph(const StepIO<S, T, A> &io, const Consts<T> &c, const Shift &sh, dim3 grid,
                           cudaStream_t st) {
    static std::atomic<unsigned long long> ready{0ull};
    cudaError_t e = allow_dynamic_smem(k_step<S, T, A, BY, PH>, stash_bytes<T, BY>(), ready);
    if (e != cudaSuccess) return e;
    e = launch_halo_ph<S, T, A, BY, PH>(io, c, sh, grid, st);
    if (e != cudaSuccess) return e;
    return launch_dependent(k_step<S, T, A, BY, PH>, grid, dim3(32, BY), stash_bytes<T, BY>(), st, io, c, sh);
}

template <typename S, typename T, typename A, int BY>
cudaError_t launch_step_by(const DevState &s, int cur, int lcur, int write_sigma, const Consts<T> &c, const Shift &sh,
                           int variant, cudaStream_t st) {
    const dim3 grid((s.nx + 31) / 32, (s.ny + BY - 1) / BY);
    const StepIO<S, T, A> io = step_io<S, T, A>(s, cur, lcur, write_sigma);
    if (variant != LBM_STEP_DIRECT) return cudaErrorInvalidValue;
    return cur ? launch_step_ph<S, T, A, BY, 1>(io, c, sh, grid, st) : launch_step_ph<S, T, A, BY, 0>(io, c, sh, grid, st);
}

template <typename S, typename T, typename A>
cudaError_t launch_step_t(const DevState &s, int cur, int lcur, int write_sigma, const void *consts, const Shift &sh,
                          int tile_rows, int variant, cudaStream_t st) {
    const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);
    switch (tile_rows) {
    case 4: return launch_step_by<S, T, A, 4>(s, cur, lcur, write_sigma, c, sh, variant, st);
    case 8: return launch_step_by<S, T, A, 8>(s, cur, lcur, write_sigma, c, sh, variant, st);
    case 16: return launch_step_by<S, T, A, 16>(s, cur, lcur, write_sigma, c, sh, variant, st);
    default: return cudaErrorInvalidValue;
    }
}

// The finish of an observation (group sums, then the observables), after
// the launch that wrote the block partials of ws.nblocks blocks.
inline cudaError_t launch_obs_finish(int nx, int ny, const ObsScratch &ws, const Scalars &sc, cudaStream_t st) {
    return launch_dependent(k_obs_finish<OBS_FINISH_THREADS>, dim3(ws.ngroups), dim3(OBS_FINISH_THREADS), 0, st, nx,
                            ny, ws, sc);
}

// The step that also reduces the observables of the state it reads.
template <typename S, typename T, typename A, int BY, int PH>
cudaError_t launch_step_obs_ph(const StepIO<S, T, A> &io, const Consts<T> &c, const Shift &sh, dim3 grid,
                               const ObsScratch &w, const Scalars &sc, cudaStream_t st) {
    static std::atomic<unsigned long long> ready{0ull};
    cudaError_t e = allow_dynamic_smem(k_step_obs<S, T, A, BY, PH>, stash_bytes<T, BY>(), ready);
    if (e != cudaSuccess) return e;
    e = launch_halo_ph<S, T, A, BY, PH>(io, c, sh, grid, st);
    if (e != cudaSuccess) return e;
    e = launch_dependent(k_step_obs<S, T, A, BY, PH>, grid, dim3(32, BY), stash_bytes<T, BY>(), st, io, c, sh, w,
                         sc);
    if (e != cudaSuccess) return e;
    return launch_obs_finish(io.nx, io.ny, w, sc, st);
}

template <typename S, typename T, typename A, int BY>
cudaError_t launch_step_obs_by(const DevState &s, int cur, int lcur, int write_sigma, const Consts<T> &c,
                               const Shift &sh, const ObsScratch &ws, const Scalars &sc, cudaStream_t st) {
    const dim3 grid((s.nx + 31) / 32, (s.ny + BY - 1) / BY);
    const StepIO<S, T, A> io = step_io<S, T, A>(s, cur, lcur, write_sigma);
    ObsScratch w = ws;
    w.nblocks = (int)(grid.x * grid.y);
    w.ngroups = (w.nblocks + OBS_GROUP - 1) / OBS_GROUP;
    return cur ? launch_step_obs_ph<S, T, A, BY, 1>(io, c, sh, grid, w, sc, st)
               : launch_step_obs_ph<S, T, A, BY, 0>(io, c, sh, grid, w, sc, st);
}

template <typename S, typename T, typename A>
cudaError_t launch_step_obs_t(const DevState &s, int cur, int lcur, int write_sigma, const void *consts,
                              const Shift &sh, int tile_rows, const ObsScratch &ws, const Scalars &sc,
                              cudaStream_t st) {
    const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);
    switch (tile_rows) {
    case 4: return launch_step_obs_by<S, T, A, 4>(s, cur, lcur, write_sigma, c, sh, ws, sc, st);
    case 8: return launch_step_obs_by<S, T, A, 8>(s, cur, lcur, write_sigma, c, sh, ws, sc, st);
    case 16: return launch_step_obs_by<S, T, A, 16>(s, cur, lcur, write_sigma, c, sh, ws, sc, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

// Batched-step entry points of one precision.
#define LBM_DEFINE_BATCH(SUFFIX, S, T, A)                                                                   \
    namespace lbm {                                                                                         \
    int batch_blocks_per_sm_##SUFFIX(int tile_rows) { return batch_blocks_per_sm_t<S, T, A>(tile_rows); }   \
    cudaError_t launch_batch_step_##SUFFIX(const BatchItem *items_dev, const void *consts_dev,             \
                                           const int *tile_item_dev, int total_tiles, int tile_rows,       \
                                           int grid, int flip_cur, int flip_l, cudaStream_t st) {          \
        return launch_batch_step_t<S, T, A>(items_dev, consts_dev, tile_item_dev, total_tiles, tile_rows,  \
                                            grid, flip_cur, flip_l, st);                                   \
    }                                                                                                       \
    cudaError_t launch_batch_sweep_##SUFFIX(const BatchItem *items_dev, const void *consts_dev, int n_items,\
                                            int total_tiles, int grid, int flip_l, int flip_cur,            \
                                            uint32_t sr_sys, cudaStream_t st) {                             \
        return launch_batch_sweep_t<S, T, A>(items_dev, consts_dev, n_items, total_tiles, grid, flip_l,     \
                                             flip_cur, sr_sys, st);                                         \
    }                                                                                                       \
    }

// ---------------------------------------------------------------------------
// Launchers for one (S, T, A) triple; SUFFIX names the precision.
// ---------------------------------------------------------------------------
#define LBM_DEFINE_LAUNCHERS(SUFFIX, S, T, A)                                                              \
    namespace lbm {                                                                                         \
    cudaError_t launch_step_##SUFFIX(const DevState &s, int cur, int lcur, int write_sigma,                 \
                                     const void *consts, const Shift &sh, int tile_rows, int variant,       \
                                     cudaStream_t st) {                                                     \
        return launch_step_t<S, T, A>(s, cur, lcur, write_sigma, consts, sh, tile_rows, variant, st);       \
    }                                                                                                       \
    cudaError_t launch_sweep_##SUFFIX(const DevState &s, int lcur, int cur, uint32_t sr_sys,               \
                                      const void *consts, const Shift &sh, cudaStream_t st) {               \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_sweep<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, lcur, cur, sr_sys, c, sh);                        \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_init_##SUFFIX(const DevState &s, const double *psi_dev, double R, double xc,        \
                                     double yc, const void *consts, const Shift &sh, cudaStream_t st) {    \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_init<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, psi_dev, R, xc, yc, double(c.W), c, sh);           \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_obs_##SUFFIX(const DevState &s, int cur, int lcur, const void *consts,              \
                                    const Shift &sh, const ObsScratch &ws, const Scalars &sc,               \
                                    cudaStream_t st) {                                                      \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        dim3 grid((s.nx + 31) / 32, (s.ny + OBS_BY - 1) / OBS_BY);                                          \
        k_obs<S, T, A><<<grid, dim3(32, OBS_BY), 0, st>>>(s, cur, lcur, c, sh, ws, sc);                     \
        const cudaError_t e = cudaGetLastError();                                                           \
        return e != cudaSuccess ? e : launch_obs_finish(s.nx, s.ny, ws, sc, st);                            \
    }                                                                                                       \
    cudaError_t launch_step_obs_##SUFFIX(const DevState &s, int cur, int lcur, int write_sigma,             \
                                         const void *consts, const Shift &sh, int tile_rows,                \
                                         const ObsScratch &ws, const Scalars &sc, cudaStream_t st) {        \
        return launch_step_obs_t<S, T, A>(s, cur, lcur, write_sigma, consts, sh, tile_rows, ws, sc, st);    \
    }                                                                                                       \
    cudaError_t launch_heat_flux_##SUFFIX(const DevState &s, int cur, int lcur, const void *consts,        \
                                          const Shift &sh, double *out, cudaStream_t st) {                  \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        k_heat_flux<S, T, A><<<(s.nx + 127) / 128, 128, 0, st>>>(s, cur, lcur, c, sh, out);                 \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_get_##SUFFIX(const DevState &s, int cur, int lcur, int field, const void *consts,   \
                                    const Shift &sh, double *out, cudaStream_t st) {                        \
        const Consts<double> &c = *reinterpret_cast<const Consts<double> *>(consts);                      \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_get<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, cur, lcur, field, c, sh, out);                      \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_phi_snap_##SUFFIX(const DevState &s, int lcur, const void *consts, const Shift &sh, \
                                         void *snap, cudaStream_t st) {                                     \
        const Consts<double> &c = *reinterpret_cast<const Consts<double> *>(consts);                      \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_phi_snap<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, lcur, c, sh, reinterpret_cast<A *>(snap));     \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_phi_change_##SUFFIX(const DevState &s, int lcur, const void *consts,                \
                                           const Shift &sh, const void *snap, unsigned long long *out,      \
                                           cudaStream_t st) {                                               \
        const Consts<double> &c = *reinterpret_cast<const Consts<double> *>(consts);                      \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_phi_change<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, lcur, c, sh, reinterpret_cast<const A *>(snap), \
                                                            out);                                           \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_place_##SUFFIX(const DevState &s, int cur, int lcur, const void *src, cudaStream_t st) { \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_place<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, cur, lcur, src);                                  \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_set_##SUFFIX(const DevState &s, int cur, int lcur, int field, const void *consts,   \
                                    const Shift &sh, const double *in, cudaStream_t st) {                   \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_set<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, cur, lcur, field, c, sh, in);                       \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    }
