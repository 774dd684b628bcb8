// Kernels of the f64 storage precision (populations double, arithmetic double, auxiliary fields double).
#include "lbm_launch.cuh"

LBM_DEFINE_LAUNCHERS(f64, double, double, double)

namespace lbm {
cudaError_t launch_batch_step_f64(const BatchItem *items_dev, const void *consts_dev, int n_items,
                                 int total_tiles, int tile_rows, int grid, int flip_cur, int flip_l,
                                 cudaStream_t st) {
    const Consts<double> *c = reinterpret_cast<const Consts<double> *>(consts_dev);
    switch (tile_rows) {
    case 4:
        {
            static bool ready = false;
            cudaError_t e = allow_dynamic_smem(k_batch_step<double, double, double, 4>, stash_bytes<double, 4>(), ready);
            if (e != cudaSuccess) return e;
        }
        k_batch_step<double, double, double, 4><<<grid, dim3(32, 4), stash_bytes<double, 4>(), st>>>(items_dev, c, n_items, total_tiles, flip_cur, flip_l);
        break;
    case 8:
        {
            static bool ready = false;
            cudaError_t e = allow_dynamic_smem(k_batch_step<double, double, double, 8>, stash_bytes<double, 8>(), ready);
            if (e != cudaSuccess) return e;
        }
        k_batch_step<double, double, double, 8><<<grid, dim3(32, 8), stash_bytes<double, 8>(), st>>>(items_dev, c, n_items, total_tiles, flip_cur, flip_l);
        break;
    case 16:
        {
            static bool ready = false;
            cudaError_t e = allow_dynamic_smem(k_batch_step<double, double, double, 16>, stash_bytes<double, 16>(), ready);
            if (e != cudaSuccess) return e;
        }
        k_batch_step<double, double, double, 16><<<grid, dim3(32, 16), stash_bytes<double, 16>(), st>>>(items_dev, c, n_items, total_tiles, flip_cur, flip_l);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
cudaError_t launch_batch_sweep_f64(const BatchItem *items_dev, const void *consts_dev, int n_items,
                                  int total_tiles, int grid, int flip_l, cudaStream_t st) {
    const Consts<double> *c = reinterpret_cast<const Consts<double> *>(consts_dev);
    k_batch_sweep<double, double, double><<<grid, dim3(32, 8), 0, st>>>(items_dev, c, n_items, total_tiles, flip_l);
    return cudaGetLastError();
}
}  // namespace lbm
