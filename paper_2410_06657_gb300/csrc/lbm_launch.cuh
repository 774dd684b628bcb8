// Host launchers of the kernels of one precision: LBM_DEFINE_LAUNCHERS(SUFFIX,
// S, T, A) defines the launch_*_SUFFIX functions declared in lbm_internal.h.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_observe.cuh"

namespace lbm {

// Resident blocks per SM of the batched step: the persistent grid is exactly
// the device's resident capacity, so every block starts at once and the
// round-robin tile share is even.
template <typename S, typename T, typename A, int BY>
int batch_blocks_per_sm_by() {
    int n = 0;
    static bool ready = false;
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
    static bool ready = false;
    cudaError_t e = allow_dynamic_smem(k_batch_step<S, T, A, BY>, stash_bytes<T, BY>(), ready);
    if (e != cudaSuccess) return e;
    k_batch_step<S, T, A, BY><<<grid, dim3(32, BY), stash_bytes<T, BY>(), st>>>(items, c, tile_item, total_tiles,
                                                                                flip_cur, flip_l);
    return cudaGetLastError();
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
                                     const void *consts, const Shift &sh, int tile_rows, cudaStream_t st) { \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        dim3 grid((s.nx + 31) / 32, (s.ny + tile_rows - 1) / tile_rows);                                   \
        const StepIO<S, T, A> io = step_io<S, T, A>(s, cur, lcur, write_sigma);                             \
        static bool r4 = false, r8 = false, r16 = false;                                                    \
        cudaError_t e = cudaSuccess;                                                                        \
        switch (tile_rows) {                                                                                \
        case 4:                                                                                             \
            e = allow_dynamic_smem(k_step<S, T, A, 4>, stash_bytes<T, 4>(), r4);                            \
            if (e == cudaSuccess)                                                                           \
                k_step<S, T, A, 4><<<grid, dim3(32, 4), stash_bytes<T, 4>(), st>>>(io, s.rng, cur, c, sh); \
            break;                                                                                          \
        case 8:                                                                                             \
            e = allow_dynamic_smem(k_step<S, T, A, 8>, stash_bytes<T, 8>(), r8);                            \
            if (e == cudaSuccess)                                                                           \
                k_step<S, T, A, 8><<<grid, dim3(32, 8), stash_bytes<T, 8>(), st>>>(io, s.rng, cur, c, sh); \
            break;                                                                                          \
        case 16:                                                                                            \
            e = allow_dynamic_smem(k_step<S, T, A, 16>, stash_bytes<T, 16>(), r16);                         \
            if (e == cudaSuccess)                                                                           \
                k_step<S, T, A, 16><<<grid, dim3(32, 16), stash_bytes<T, 16>(), st>>>(io, s.rng, cur, c, sh); \
            break;                                                                                          \
        default: return cudaErrorInvalidValue;                                                              \
        }                                                                                                   \
        if (e != cudaSuccess) return e;                                                                     \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    size_t tma_smem_##SUFFIX(int tile_rows) {                                                              \
        switch (tile_rows) {                                                                                \
        case 4: return TmaGeom<S, A, 4>::total + 128;                                                       \
        case 8: return TmaGeom<S, A, 8>::total + 128;                                                       \
        case 16: return TmaGeom<S, A, 16>::total + 128;                                                     \
        default: return 0;                                                                                  \
        }                                                                                                   \
    }                                                                                                       \
    template <int BY>                                                                                       \
    static cudaError_t launch_tma_by_##SUFFIX(const DevState &s, int cur, int lcur, int write_sigma,        \
                                              const Consts<T> &c, const Shift &sh, const TmaMaps &m,        \
                                              cudaStream_t st) {                                            \
        if constexpr (!std::is_same<typename FStore<S>::type, S>::value) {                                  \
            return cudaErrorNotSupported;         /* the tensor boxes assume one storage type */            \
        } else {                                                                                            \
            static bool ready = false;                                                                      \
            if (!ready) {                                                                                   \
                cudaError_t e = cudaFuncSetAttribute(k_step_tma<S, T, A, BY>,                               \
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                                     (int)TmaGeom<S, A, BY>::total + 128);                  \
                if (e != cudaSuccess) return e;                                                             \
                ready = true;                                                                               \
            }                                                                                               \
            dim3 grid((s.nx + 31) / 32, (s.ny + BY - 1) / BY);                                              \
            k_step_tma<S, T, A, BY><<<grid, dim3(32, BY), TmaGeom<S, A, BY>::total + 128, st>>>(            \
                s, cur, lcur, write_sigma, c, sh, m.fhg[cur], m.l[lcur], m.aux[cur]);                       \
            return cudaGetLastError();                                                                      \
        }                                                                                                   \
    }                                                                                                       \
    cudaError_t launch_step_tma_##SUFFIX(const DevState &s, int cur, int lcur, int write_sigma,             \
                                         const void *consts, const Shift &sh, const TmaMaps &m,             \
                                         cudaStream_t st) {                                                 \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        switch (m.by) {                                                                                     \
        case 4: return launch_tma_by_##SUFFIX<4>(s, cur, lcur, write_sigma, c, sh, m, st);                  \
        case 8: return launch_tma_by_##SUFFIX<8>(s, cur, lcur, write_sigma, c, sh, m, st);                  \
        case 16: return launch_tma_by_##SUFFIX<16>(s, cur, lcur, write_sigma, c, sh, m, st);                \
        default: return cudaErrorInvalidValue;                                                              \
        }                                                                                                   \
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
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    cudaError_t launch_step_obs_##SUFFIX(const DevState &s, int cur, int lcur, int write_sigma,             \
                                         const void *consts, const Shift &sh, int tile_rows,                \
                                         const ObsScratch &ws, const Scalars &sc, cudaStream_t st) {        \
        const Consts<T> &c = *reinterpret_cast<const Consts<T> *>(consts);                                \
        dim3 grid((s.nx + 31) / 32, (s.ny + tile_rows - 1) / tile_rows);                                   \
        const StepIO<S, T, A> io = step_io<S, T, A>(s, cur, lcur, write_sigma);                             \
        ObsScratch w = ws;                                                                                  \
        w.nblocks = (int)(grid.x * grid.y);                                                                 \
        w.ngroups = (w.nblocks + OBS_GROUP - 1) / OBS_GROUP;                                                \
        static bool r4 = false, r8 = false, r16 = false;                                                    \
        cudaError_t e = cudaSuccess;                                                                        \
        switch (tile_rows) {                                                                                \
        case 4:                                                                                             \
            e = allow_dynamic_smem(k_step_obs<S, T, A, 4>, stash_bytes<T, 4>(), r4);                        \
            if (e == cudaSuccess)                                                                           \
                k_step_obs<S, T, A, 4><<<grid, dim3(32, 4), stash_bytes<T, 4>(), st>>>(                     \
                    io, s.rng, cur, c, sh, w, sc);                                                          \
            break;                                                                                          \
        case 8:                                                                                             \
            e = allow_dynamic_smem(k_step_obs<S, T, A, 8>, stash_bytes<T, 8>(), r8);                        \
            if (e == cudaSuccess)                                                                           \
                k_step_obs<S, T, A, 8><<<grid, dim3(32, 8), stash_bytes<T, 8>(), st>>>(                     \
                    io, s.rng, cur, c, sh, w, sc);                                                          \
            break;                                                                                          \
        case 16:                                                                                            \
            e = allow_dynamic_smem(k_step_obs<S, T, A, 16>, stash_bytes<T, 16>(), r16);                     \
            if (e == cudaSuccess)                                                                           \
                k_step_obs<S, T, A, 16><<<grid, dim3(32, 16), stash_bytes<T, 16>(), st>>>(                  \
                    io, s.rng, cur, c, sh, w, sc);                                                          \
            break;                                                                                          \
        default: return cudaErrorInvalidValue;                                                              \
        }                                                                                                   \
        if (e != cudaSuccess) return e;                                                                     \
        return cudaGetLastError();                                                                          \
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
    cudaError_t launch_phi_change_##SUFFIX(const DevState &s, int la, int lb, const void *consts,         \
                                           const Shift &sh, unsigned long long *out, cudaStream_t st) {     \
        const Consts<double> &c = *reinterpret_cast<const Consts<double> *>(consts);                      \
        dim3 grid((s.nx + 31) / 32, (s.ny + 7) / 8);                                                        \
        k_phi_change<S, T, A><<<grid, dim3(32, 8), 0, st>>>(s, la, lb, c, sh, out);                         \
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
