// Observables of a caller-held state with no device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a runtime which
// has already reserved the device's memory for its own pool (an allocation
// here would fail or fragment that pool), and latency-critical loops where
// cudaMalloc/cudaFree would synchronise the device and stall other streams.
// For them the reduction behind lbm_observables is offered with its scratch
// (block partial sums and the crossing candidates) in a fixed-size array in
// the module's own device memory.  Every GPU that loads the library holds
// this array until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbm_internal.h"

namespace {

constexpr int kMaxBlocks = 20480;   // 32 x 8 tiles of the reduction grid
constexpr int kMaxNy = 4096;        // rows (one crossing slot per row)

constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr int kMaxGroups = (kMaxBlocks + lbm::OBS_GROUP - 1) / lbm::OBS_GROUP;
constexpr size_t kPartBytes = al256(size_t(kMaxBlocks + kMaxGroups) * lbm::OBS_NSUM * sizeof(double));
constexpr size_t kMaxvBytes = al256(size_t(2 + kMaxNy) * sizeof(unsigned long long));
constexpr size_t kMinvBytes = al256(size_t(1 + kMaxNy) * sizeof(unsigned long long));
constexpr size_t kU32Bytes = al256(size_t(kMaxNy + 3 + kMaxGroups) * sizeof(unsigned int));
constexpr size_t kScratchBytes = kPartBytes + kMaxvBytes + kMinvBytes + kU32Bytes;   // about 1.3 MB

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_dev[kMaxDevices] = {};   // last looked-up device address of the array, per device

}  // namespace

// The scratch array.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_obs_scratch[kScratchBytes];

namespace {

// Device address of the scratch array on the current device.  The address is
// looked up on every call (a device reset or a new primary context reloads
// the module, which moves the array); only while `st` is being captured into
// a graph, where a lookup could load a module, the value of the last lookup
// on this device is used, and a capture before any lookup is refused.
int scratch_address(cudaStream_t st, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        lbm::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        lbm::set_last_error("device ordinal beyond the supported range");
        return LBM_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) {
        lbm::set_last_error(std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs != cudaStreamCaptureStatusNone) {
        if (!g_scratch_dev[dev]) {
            lbm::set_last_error("the first call on a device must come before any stream capture");
            return LBM_ERR_CUDA;
        }
        *out = g_scratch_dev[dev];
        return LBM_OK;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_obs_scratch);
    if (e != cudaSuccess || !p) {
        lbm::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    g_scratch_dev[dev] = p;
    *out = p;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_observables_noalloc(const lbm_params *p, const void *pop, const void *aux, int32_t pitch,
                                       int64_t step, lbm_obs *out, void *stream) {
    using namespace lbm;
    if (!p || !pop || !aux || !out) {
        set_last_error("NULL argument");
        return LBM_ERR_BADPARAM;
    }
    Consts<double> cd;
    Consts<float> cf;
    Shift sh;
    const char *why = nullptr;
    if (derive_for_noalloc(p, &cd, &cf, &sh, &why) != LBM_OK) {
        set_last_error(why ? why : "invalid parameters");
        return LBM_ERR_BADPARAM;
    }
    const int nblocks = obs_blocks(p->nx, p->ny);
    if (p->ny > kMaxNy || nblocks > kMaxBlocks) {
        set_last_error("lattice beyond the fixed scratch: at most 4096 rows and 20480 tiles of 32 x 8 cells");
        return LBM_ERR_BADPARAM;
    }
    if (pitch < p->nx) {
        set_last_error("pitch must be at least nx");
        return LBM_ERR_BADPARAM;
    }
    // the kernel reads every plane element by element: both arrays must be
    // aligned to the widest element they hold, and so must the result
    const uintptr_t pop_align = p->precision == LBM_FP64 ? 8 : 4, aux_align = pop_align;
    if (reinterpret_cast<uintptr_t>(pop) % pop_align || reinterpret_cast<uintptr_t>(aux) % aux_align ||
        reinterpret_cast<uintptr_t>(out) % alignof(lbm_obs)) {
        set_last_error("pop, aux and out must be aligned to their element size (8 bytes for FP64 and lbm_obs, "
                       "4 for FP32 and half storage)");
        return LBM_ERR_BADPARAM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    int rc = scratch_address(st, &base);
    if (rc != LBM_OK) return rc;

    unsigned char *b = static_cast<unsigned char *>(base);
    ObsScratch ws;
    ws.partials = reinterpret_cast<double *>(b);
    ws.maxv = reinterpret_cast<unsigned long long *>(b + kPartBytes);
    ws.minv = reinterpret_cast<unsigned long long *>(b + kPartBytes + kMaxvBytes);
    ws.rowany = reinterpret_cast<unsigned int *>(b + kPartBytes + kMaxvBytes + kMinvBytes);
    ws.bad = ws.rowany + p->ny;
    ws.gcount = ws.rowany + p->ny + 3;
    ws.ngroups = (nblocks + OBS_GROUP - 1) / OBS_GROUP;
    ws.gpartials = ws.partials + (size_t)nblocks * OBS_NSUM;
    ws.obs = out;
    ws.nblocks = nblocks;

    DevState s;
    s.pop = const_cast<void *>(pop);          // natural layout (phase 0)
    s.aux[0] = s.aux[1] = const_cast<void *>(aux);
    s.sigma = nullptr;
    s.halo = nullptr;
    s.err = nullptr;
    s.rng = nullptr;
    s.nx = p->nx;
    s.ny = p->ny;
    s.pitch = pitch;
    s.plane = (long long)pitch * p->ny;

    Scalars sc;
    sc.step = step;
    sc.alpha_l = p->alpha_l;
    sc.R0 = p->R0;

    // the array keeps the previous call's contents: reset what must start
    // at the identity of its reduction (0 for maxima and flags, all ones for
    // minima)
    cudaError_t e = cudaMemsetAsync(ws.maxv, 0x00, (size_t)(2 + p->ny) * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.minv, 0xFF, (size_t)(1 + p->ny) * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.rowany, 0x00, (size_t)(p->ny + 3 + ws.ngroups) * sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        switch (p->precision) {
        case LBM_FP64: e = launch_obs_f64(s, 0, 0, &cd, sh, ws, sc, st); break;
        case LBM_FP32: e = launch_obs_f32(s, 0, 0, &cf, sh, ws, sc, st); break;
        default: e = launch_obs_f16s(s, 0, 0, &cf, sh, ws, sc, st); break;
        }
    }
    if (e != cudaSuccess) {
        set_last_error(std::string("observables launch: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
