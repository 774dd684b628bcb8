// The stochastic rounding of half storage on its own, for checking the
// conversion the half-storage step uses against its definition.  Built with
// the half-storage step's flags, from the same device function.
#include "lbm_kernels.cuh"

namespace lbm {

// One value per thread of a grid-stride loop, with the caller's random bits.
__global__ void k_round_half_sr(const float *__restrict__ v, const uint32_t *__restrict__ r,
                                uint16_t *__restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __half_as_ushort(half_sr(v[i], r[i] & 0x1fffu));
}

cudaError_t launch_round_half_sr(const float *v, const uint32_t *r, uint16_t *out, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    k_round_half_sr<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(v, r, out, n);
    return cudaGetLastError();
}

}  // namespace lbm
