// Observables, the substrate heat flux and field access of the
// phase-field LB electrofreezing step (arXiv 2410.06657), templated like
// the step kernels in lbm_kernels.cuh (storage type S, arithmetic type T,
// auxiliary type A).  Included once by each precision's translation unit,
// after lbm_kernels.cuh.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Observables: FP64 reductions over the tile grid.  Each block
// handles a 32 x 8 tile plus a one-cell halo (for q_v's stencils and the
// interface crossings) and leaves block partial sums and order-independent
// max/min candidates in the workspace; the last block of each group of
// OBS_GROUP blocks sums its group and the last group finishes the reduction.
// ---------------------------------------------------------------------------
constexpr int OBS_BY = 8;

// Counter increment with acquire-release semantics at GPU scope.  One
// thread increments after a block barrier: the release covers every write
// the block made before the barrier (its partials, its atomics), and the
// block that draws the last count acquires all of them, then shares them
// with its other threads through the next barrier; no thread needs a fence
// of its own.
static __device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

static __device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double v) {
    atomicMax(a, (unsigned long long)__double_as_longlong(v));   // v >= 0: bits order like values
}
static __device__ __forceinline__ void atomic_min_pos(unsigned long long *a, double v) {
    atomicMin(a, (unsigned long long)__double_as_longlong(v));
}

// An instance's populations read through the in-place layout of phases
// (ph, lph) (the AA pattern of lbm_kernels.cuh): offsets of the slot that
// holds population i of cell (x, y).
template <typename S>
struct PopView {
    Planes<S> pl;
    int ph, lph, nx, ny;
    uint32_t P, pitch;
    __host__ __device__ static PopView at(const DevState &s, int cur, int lcur) {
        PopView v;
        v.pl = Planes<S>::at(s.pop, s.plane);
        v.ph = cur;
        v.lph = lcur;
        v.nx = s.nx;
        v.ny = s.ny;
        v.P = (uint32_t)s.plane;
        v.pitch = (uint32_t)s.pitch;
        return v;
    }
    __device__ __forceinline__ uint32_t o9(int i, int x, int y) const {
        return aa_src<9>(ph, i, P, pitch, x, y, x == 0 ? nx - 1 : x - 1, x == nx - 1 ? 0 : x + 1, ny);
    }
    __device__ __forceinline__ uint32_t o5(int i, int x, int y) const {
        return aa_src<5>(lph, i, P, pitch, x, y, x == 0 ? nx - 1 : x - 1, x == nx - 1 ? 0 : x + 1, ny);
    }
};

template <typename S, typename T, typename A>
__device__ __forceinline__ void obs_macros(const PopView<S> &v, const A *aux, int x, int y,
                                           const Consts<double> &c, const Shift &sh, Macro<double> &m) {
    Refs<T> rf;
    Consts<T> ct;      // only phi_bot/phi_top/ny are used by make_refs
    ct.phi_bot = T(c.phi_bot);
    ct.phi_top = T(c.phi_top);
    make_refs<S, T>(rf, sh, ct, y, v.ny);
    const uint32_t k = (uint32_t)y * v.pitch + (uint32_t)x;
    double f[9], g[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const uint32_t o = v.o9(i, x, y);
        f[i] = double(Pol<typename FStore<S>::type, T>::ld(v.pl.f + o, rf.f[i], 1.0f / sh.f_scale));
        g[i] = double(Pol<S, T>::ld(v.pl.g + o, rf.g[i], 1.0f / sh.g_scale));
    }
    double l1234 = 0.0;
#pragma unroll
    for (int i = 1; i < 5; i++) l1234 += double(Pol<S, T>::ld(v.pl.l + v.o5(i, x, y), rf.l[i], 1.0f / sh.l_scale));
    local_macros<double>(f, g, l1234, double(aux[AUX_FS * v.P + k]), double(aux[AUX_MDOT * v.P + k]),
                         double(aux[AUX_Q * v.P + k]), c, m);
}


template <typename S, typename T, typename A>
__device__ __forceinline__ void load_cell(const PopView<S> &v, const A *aux, int x, int y, const Consts<T> &c,
                                          const Shift &sh, CellLoad<T> &o) {
    Refs<T> rf;
    make_refs<S, T>(rf, sh, c, y, v.ny);
    const uint32_t k = (uint32_t)y * v.pitch + (uint32_t)x;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const uint32_t oo = v.o9(i, x, y);
        o.f[i] = Pol<typename FStore<S>::type, T>::ld(v.pl.f + oo, rf.f[i], 1.0f / sh.f_scale);
        o.g[i] = Pol<S, T>::ld(v.pl.g + oo, rf.g[i], 1.0f / sh.g_scale);
    }
    o.l1234 = T(0);
#pragma unroll
    for (int i = 1; i < 5; i++) o.l1234 += Pol<S, T>::ld(v.pl.l + v.o5(i, x, y), rf.l[i], 1.0f / sh.l_scale);
    o.fs_prev = T(aux[AUX_FS * v.P + k]);
    o.mdot_prev = T(aux[AUX_MDOT * v.P + k]);
    o.Q_prev = T(aux[AUX_Q * v.P + k]);
}

// Local macros of one cell in the arithmetic type T (the step's own type).
template <typename S, typename T, typename A>
__device__ __forceinline__ void cell_macros_t(const PopView<S> &v, const A *aux, int x, int y, const Consts<T> &c,
                                              const Shift &sh, Macro<T> &m) {
    CellLoad<T> o;
    load_cell<S, T, A>(v, aux, x, y, c, sh, o);
    local_macros<T>(o.f, o.g, o.l1234, o.fs_prev, o.mdot_prev, o.Q_prev, c, m);
}

template <int NT>
static __device__ __forceinline__ void obs_final(int nx, int ny, const ObsScratch &ws, const Scalars &sc);

// Sum of n values of quantity j at src[i * OBS_NSUM + j] (i < n), by one warp
// in a fixed order: lane l adds i = l, l + 32, ..., then a butterfly of
// shuffles.  Every lane returns the sum; lane 0 stores it in *out32.
static __device__ __forceinline__ double warp_sum_fixed(const double *src, int n, int j, double *out32) {
    const int lane = threadIdx.x & 31;
    double v = lane < n ? __ldcg(src + (long long)lane * OBS_NSUM + j) : 0.0;
    for (int i = lane + 32; i < n; i += 32) v += __ldcg(src + (long long)i * OBS_NSUM + j);
#pragma unroll
    for (int h = 16; h > 0; h >>= 1) v += __shfl_xor_sync(0xffffffffu, v, h);
    if (lane == 0) out32[0] = v;
    return v;
}

// First level: block g of the finish launch sums group g's block partials
// (warp w sums quantities w, w + NT/32, ...).
template <int NT>
static __device__ __forceinline__ void obs_group(const ObsScratch &ws, int g, int gsize) {
    __shared__ double s_g[OBS_NSUM][32];
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < OBS_NSUM; j += NT / 32) {
        const double v = warp_sum_fixed(ws.partials + (long long)g * OBS_GROUP * OBS_NSUM, gsize, j, s_g[j]);
        if (lane == 0) ws.gpartials[(long long)g * OBS_NSUM + j] = v;
    }
}

// The end of one block's part of the reduction (NT threads, one warp per
// lattice row y): row flags and the block sums (warp sums in R, warps
// combined in FP64 in a fixed order), written as the block's partials.
// The finish is a launch of its own (k_obs_finish), so the blocks of the
// reducing kernel end without a fence or a counter.
template <int NT, typename R>
static __device__ __forceinline__ void obs_block_finish(const ObsScratch &ws, const R (&v)[OBS_NSUM],
                                                        unsigned int rowbits, int y, int ny) {
    __shared__ double s_red[OBS_NSUM][NT / 32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    // row flags: OR across the warp (all lanes share the row), one atomic
    {
        unsigned int b = rowbits;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b |= __shfl_xor_sync(0xffffffffu, b, o);
        if (tx == 0 && b && y < ny) atomicOr(&ws.rowany[y], b);
    }
#pragma unroll
    for (int j = 0; j < OBS_NSUM; j++) {
        R t = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (tx == 0) s_red[j][ty] = double(t);
    }
    __syncthreads();
    if (tid < OBS_NSUM) {
        double t = s_red[tid][0];
        for (int w = 1; w < NT / 32; w++) t += s_red[tid][w];
        ws.partials[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * OBS_NSUM + tid] = t;
    }
}

// The two-level finish of an observation, after the kernel that wrote the
// block partials (its grid of ws.nblocks blocks).  FP64 adds run at a small
// fraction of the FP32 rate on this part, so they are spread over many SMs:
// block g of this launch (ws.ngroups blocks of NT threads) sums group g of
// OBS_GROUP block partials, and the last of them to finish sums the groups
// and writes the observables.  Every sum runs in a fixed order.
template <int NT>
__global__ void __launch_bounds__(NT) k_obs_finish(int nx, int ny, ObsScratch ws, Scalars sc) {
    grid_dep_wait();                   // the partials, crossings and flags of the reducing kernel
    grid_dep_release();
    const int g = blockIdx.x, gsize = min(OBS_GROUP, ws.nblocks - g * OBS_GROUP);
    obs_group<NT>(ws, g, gsize);
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = atom_add_acq_rel(ws.bad + 2, 1u) == (unsigned int)ws.ngroups - 1u;
    __syncthreads();
    if (s_last) obs_final<NT>(nx, ny, ws, sc);
}
constexpr int OBS_FINISH_THREADS = 256;      // a warp per quantity

template <typename S, typename T, typename A>
__global__ void __launch_bounds__(32 * OBS_BY) k_obs(DevState s, int cur, int lcur, Consts<T> c, Shift sh,
                                                    ObsScratch ws, Scalars sc) {
    // per-cell values and the q_v stencils in the step's arithmetic; sums
    // within a warp in the step's type (FP64 adds are slow on this part;
    // a 32-term sum of single-precision values loses ~1e-7), across warps
    // and blocks in FP64; interface crossings and the front in FP64
    using R = typename std::conditional<sizeof(T) == 8, double, float>::type;
    __shared__ T s_psi[OBS_BY + 2][34], s_fs[OBS_BY + 2][34], s_eps[OBS_BY + 2][34], s_phi[OBS_BY + 2][34];
    __shared__ T s_H[OBS_BY + 2][34], s_Tm[OBS_BY + 2][34];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int nx = s.nx, ny = s.ny;
    const long long P = s.plane;
    const PopView<S> pv = PopView<S>::at(s, cur, lcur);
    const A *aux = reinterpret_cast<const A *>(cur ? s.aux[1] : s.aux[0]);
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * OBS_BY;
    // fill the extended tile (own + halo), ghost rows as in the step: each
    // thread takes at most two of the 34 x (OBS_BY + 2) cells and issues the
    // loads of both before evaluating either
    static_assert(34 * (OBS_BY + 2) <= 2 * 32 * OBS_BY, "two cells per thread");
    {
        CellLoad<T> ld[2];
        int slot_ex[2], slot_ey[2];
        bool valid[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int r = tid + q * 32 * OBS_BY;
            slot_ex[q] = r % 34;
            slot_ey[q] = r / 34;
            const int yy = y0 - 1 + slot_ey[q];
            valid[q] = r < 34 * (OBS_BY + 2) && yy >= 0 && yy < ny;
            if (valid[q]) {
                int xx = x0 - 1 + slot_ex[q];
                xx = xx < 0 ? xx + nx : (xx >= nx ? (xx - nx < nx ? xx - nx : (xx - nx) % nx) : xx);
                load_cell<S, T, A>(pv, aux, xx, yy, c, sh, ld[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            if (!valid[q]) continue;
            Macro<T> m;
            local_macros<T>(ld[q].f, ld[q].g, ld[q].l1234, ld[q].fs_prev, ld[q].mdot_prev, ld[q].Q_prev, c, m);
            const int ex = slot_ex[q], ey = slot_ey[q];
            s_psi[ey][ex] = m.psi;
            s_fs[ey][ex] = m.fs;
            s_eps[ey][ex] = m.eps;
            s_phi[ey][ex] = m.phi;
            s_H[ey][ex] = m.H;
            s_Tm[ey][ex] = m.T_;
        }
    }
    __syncthreads();
    if (y0 == 0 && tid < 34) {
        s_eps[0][tid] = s_eps[1][tid];
        s_phi[0][tid] = T(2) * c.phi_bot - s_phi[1][tid];
    }
    const int et = ny - y0 + 1;
    if (et >= 1 && et <= OBS_BY + 1 && tid >= 64 && tid < 98) {
        s_eps[et][tid - 64] = s_eps[et - 1][tid - 64];
        s_phi[et][tid - 64] = T(2) * c.phi_top - s_phi[et - 1][tid - 64];
    }
    __syncthreads();

    const int x = x0 + tx, y = y0 + ty;
    R v_psi = R(0), v_H = R(0), v_fs = R(0), v_q = R(0), v_liq = R(0), v_liqu = R(0), v_qdot = R(0);
    unsigned int rowbits = 0u;                // this lane's row flags (one warp = one row)
    if (x < nx && y < ny) {
        const int ex = tx + 1, ey = ty + 1;
        Macro<T> m;                           // this cell's values, from the extended tile
        m.psi = s_psi[ey][ex];
        m.fs = s_fs[ey][ex];
        m.eps = s_eps[ey][ex];
        m.H = s_H[ey][ex];
        const long long k = (long long)y * s.pitch + x;
        // substrate heat flux (R24): -k (4 T_1 - T_2 - 3 T_0) / 2 on row 0
        if (y == 0 && ny >= 3) {
            const T kth0 = chi(m.fs, m.psi, c.kth);
            v_qdot = R(-kth0 * (T(4) * s_Tm[2][ex] - s_Tm[3][ex] - T(3) * s_Tm[1][ex]) / T(2));
        }
        // Peclet number (R25): liquid content psi - f_s weights |psi u| / psi
        {
            const T w = m.psi - m.fs;
            if (w > T(0)) {
                const T ux = T(aux[AUX_PUX * P + k]), uy = T(aux[AUX_PUY * P + k]);
                const T sp = sqrt(ux * ux + uy * uy);
                v_liq = R(w);
                v_liqu = R(w * sp / m.psi);
            }
        }
        T gex, gey, gphx, gphy;
        constexpr bool RED = reduced_stencils<S>();
        grad_s<T, 34, RED>(s_eps, ex, ey, gex, gey);
        grad_s<T, 34, RED>(s_phi, ex, ey, gphx, gphy);
        const T lphi = lap_s<T, 34, RED>(s_phi, ex, ey);
        v_q = R(-(gex * gphx + gey * gphy + m.eps * lphi));
        v_psi = R(m.psi);
        v_H = R(m.H);
        v_fs = R(m.fs);
        if (!isfinite(v_psi) || !isfinite(v_H)) atomicOr(ws.bad, 1u);
        const double a = double(s_psi[ey][ex]);
        // column crossing (height): psi(y) >= 1/2 > psi(y+1)
        if (a >= 0.5) {
            rowbits |= 1u;
            if (y == ny - 1) {
                atomic_max_pos(&ws.maxv[0], (double)ny);
            } else {
                const double b = double(s_psi[ey + 1][ex]);
                if (b < 0.5) atomic_max_pos(&ws.maxv[0], y + (a - 0.5) / (a - b) + 0.5);
            }
            // row crossings (width): left edge needs x >= 1, right edge x <= nx - 2
            if (x >= 1) {
                const double bl = double(s_psi[ey][ex - 1]);
                if (bl < 0.5) {
                    atomic_min_pos(&ws.minv[1 + y], (x - 1) + (0.5 - bl) / (a - bl));
                    rowbits |= 2u;
                }
            }
            if (x + 1 < nx) {
                const double br = double(s_psi[ey][ex + 1]);
                if (br < 0.5) {
                    atomic_max_pos(&ws.maxv[2 + y], x + (a - 0.5) / (a - br));
                    rowbits |= 4u;
                }
            }
        }
        // freezing front on the centre column (lowest f_s = 1/2 crossing)
        if (x == nx / 2) {
            const double fa = double(s_fs[ey][ex]);
            if (y == 0 && fa >= 0.5) atomicOr(ws.bad + 1, 1u);
            if (fa >= 0.5) {
                if (y == ny - 1) {
                    atomic_min_pos(&ws.minv[0], (double)ny);
                } else {
                    const double fb = double(s_fs[ey + 1][ex]);
                    if (fb < 0.5) atomic_min_pos(&ws.minv[0], y + (fa - 0.5) / (fa - fb) + 0.5);
                }
            }
        }
    }
    const R v[OBS_NSUM] = {v_psi, v_H, v_fs, v_q, v_liq, v_liqu, v_qdot};
    obs_block_finish<32 * OBS_BY, R>(ws, v, rowbits, y, ny);
}

// psi = 1/2 extent of row y: 0 without liquid, nx without a left or right
// crossing (the row is liquid across the periodic seam), else right - left.
// (Other blocks wrote the workspace with atomics during this launch: read
// it from L2.)
static __device__ __forceinline__ double row_extent_of(const ObsScratch &ws, int y, int nx) {
    // the three loads are independent: one round trip
    const unsigned int bits = __ldcg(ws.rowany + y);
    const unsigned long long r = __ldcg(ws.maxv + 2 + y), l = __ldcg(ws.minv + 1 + y);
    if (!(bits & 1u)) return 0.0;
    if ((bits & 6u) != 6u) return (double)nx;
    return __longlong_as_double((long long)r) - __longlong_as_double((long long)l);
}

// Final reduction, run by the last group to finish (NT >= 128 threads): the
// group sums in a fixed order, the widest row, the single values and the
// result, so nothing depends on which block finishes last.
template <int NT>
static __device__ __forceinline__ void obs_final(int nx, int ny, const ObsScratch &ws, const Scalars &sc) {
    static_assert(NT >= 128 && NT % 32 == 0, "four warps at least");
    __shared__ double s_height, s_rtr, s_front;
    __shared__ unsigned int s_bad;
    __shared__ long long s_tfre;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    // the single values, by the last warp, while the sums are gathered
    if (t == NT - 32) {
        s_height = __longlong_as_double((long long)__ldcg(ws.maxv));
        const unsigned long long fmin = __ldcg(ws.minv);
        s_front = __ldcg(ws.bad + 1) ? ((fmin == ~0ull) ? (double)ny : __longlong_as_double((long long)fmin)) : 0.0;
        s_bad = __ldcg(ws.bad);
        s_tfre = (long long)__ldcg(&ws.obs->t_fre);
        s_rtr = 0.5 * row_extent_of(ws, 0, nx);
    }
    // the group sums (warp w sums quantities w, w + NT/32, ... over the groups)
    __shared__ double s_fin[OBS_NSUM][32];
    for (int j = t >> 5; j < OBS_NSUM; j += NT / 32) warp_sum_fixed(ws.gpartials, ws.ngroups, j, s_fin[j]);
    // widest row: extents are non-negative doubles, so their bit patterns
    // order like the values and the maximum is an integer one
    __shared__ unsigned long long s_wb[NT / 32];
    unsigned long long wb = 0ull;
    for (int y = t; y < ny; y += NT) {
        const unsigned long long e = (unsigned long long)__double_as_longlong(row_extent_of(ws, y, nx));
        wb = e > wb ? e : wb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, wb, o);
        wb = other > wb ? other : wb;
    }
    if ((t & 31) == 0) s_wb[t >> 5] = wb;
    __syncthreads();
    // everything from registers and shared memory; the FP64 divisions are
    // long on this part, so four warps take one group of results each
    lbm_obs *o = ws.obs;
    if (t == 0) {
        const double mass = s_fin[0][0], solid = s_fin[2][0];
        const double ff = (mass != 0.0) ? solid / mass : 0.0;
        long long t_fre = s_tfre;
        if (t_fre < 0 && ff >= 0.99) t_fre = sc.step;
        o->step = sc.step;
        o->mass = mass;
        o->enthalpy = s_fin[1][0];
        o->solid = solid;
        o->charge = s_fin[3][0];
        o->frozen_fraction = ff;
        o->R_tr = s_rtr;
        o->front = s_front;
        o->t_fre = t_fre;
        o->Fo_fre = (t_fre >= 0) ? sc.alpha_l * (double)t_fre / (sc.R0 * sc.R0) : -1.0;
        o->status = s_bad ? LBM_ERR_DIVERGED : LBM_OK;
        o->reserved = 0;
        o->Qdot = s_fin[6][0];                                                  // R24
    } else if (t == 32) {
        o->Fo = sc.alpha_l * (double)sc.step / (sc.R0 * sc.R0);
    } else if (t == 64) {
        unsigned long long wmax = s_wb[0];
        for (int w = 1; w < NT / 32; w++) wmax = s_wb[w] > wmax ? s_wb[w] : wmax;
        const double width = __longlong_as_double((long long)wmax), height = s_height;
        o->height = height;
        o->width = width;
        o->aspect = (width > 0.0) ? height / width : 0.0;
    } else if (t == 96) {
        const double liq = s_fin[4][0], liqu = s_fin[5][0];
        o->Pe = (liq > 0.0) ? 2.0 * sc.R0 * (liqu / liq) / sc.alpha_l : 0.0;     // R25
    }
    // leave the workspace at the identities of its reductions for the next
    // call (0 for maxima and flags, all ones for minima)
    __syncthreads();
    for (int i = t; i < ny + 2; i += NT) ws.maxv[i] = 0ull;
    for (int i = t; i < ny + 1; i += NT) ws.minv[i] = ~0ull;
    for (int i = t; i < ny + 3; i += NT) ws.rowany[i] = 0u;     // rowany[ny], then bad[0..2]
}

// ---------------------------------------------------------------------------
// Observables fused into a step.  The step from time n to n + 1 reads the
// state at time n and already evaluates, for its tile and the ring around
// it, every macro the observables need (and q_v with the same stencils), so
// an observation of the state at time n can ride on that step instead of
// reading the lattice once more.  The terms and crossings are k_obs's; the
// step's 32 x BY tile (one warp per row) replaces k_obs's 32 x 8 one, so the
// FP64 sums group the same terms differently (rounding only).
// ---------------------------------------------------------------------------
template <typename T, int BY>
struct StepObs {
    using R = typename std::conditional<sizeof(T) == 8, double, float>::type;
    T (*fs)[34];                  // f_s of the extended tile (shared memory)
    T (*Tm)[34];                  // temperature of the extended tile (shared memory)
    unsigned long long *maxv, *minv;
    unsigned int *bad;
    R v[OBS_NSUM];                // psi, H, f_s, q_v, liquid, liquid speed, Qdot of the own cell
    unsigned int rowbits;         // bit0 liquid, bit1 left crossing, bit2 right crossing

    __device__ __forceinline__ void macro(int ey, int ex, const Macro<T> &m) {
        fs[ey][ex] = m.fs;
        Tm[ey][ex] = m.T_;
    }

    template <typename S, typename A>
    __device__ __forceinline__ void cell(const StepIO<S, T, A> &io, const Consts<T> &c, const TileSmem<T, BY> &sm,
                                         int tx, int ty, int x, int y, uint32_t k, const Macro<T> &m, T qv) {
        const int ex = tx + 1, ey = ty + 1, nx = io.nx, ny = io.ny;
        const uint32_t P = (uint32_t)io.plane;
        // substrate heat flux (R24): -k (4 T_1 - T_2 - 3 T_0) / 2 on row 0
        if (y == 0 && ny >= 3) {
            const T kth0 = chi(m.fs, m.psi, c.kth);
            v[6] = R(-kth0 * (T(4) * Tm[2][ex] - Tm[3][ex] - T(3) * Tm[1][ex]) / T(2));
        }
        // Peclet number (R25): liquid content psi - f_s weights |psi u| / psi
        {
            const T w = m.psi - m.fs;
            if (w > T(0)) {
                const T ux = T(io.aux_in[AUX_PUX * P + k]), uy = T(io.aux_in[AUX_PUY * P + k]);
                const T sp = sqrt(ux * ux + uy * uy);
                v[4] = R(w);
                v[5] = R(w * sp / m.psi);
            }
        }
        v[3] = R(qv);
        v[0] = R(m.psi);
        v[1] = R(m.H);
        v[2] = R(m.fs);
        if (!isfinite(v[0]) || !isfinite(v[1])) atomicOr(bad, 1u);
        const double a = double(m.psi);
        // column crossing (height): psi(y) >= 1/2 > psi(y+1)
        if (a >= 0.5) {
            rowbits |= 1u;
            if (y == ny - 1) {
                atomic_max_pos(&maxv[0], (double)ny);
            } else {
                const double b = double(sm.q[ey + 1][ex].psi);
                if (b < 0.5) atomic_max_pos(&maxv[0], y + (a - 0.5) / (a - b) + 0.5);
            }
            // row crossings (width): left edge needs x >= 1, right edge x <= nx - 2
            if (x >= 1) {
                const double bl = double(sm.q[ey][ex - 1].psi);
                if (bl < 0.5) {
                    atomic_min_pos(&minv[1 + y], (x - 1) + (0.5 - bl) / (a - bl));
                    rowbits |= 2u;
                }
            }
            if (x + 1 < nx) {
                const double br = double(sm.q[ey][ex + 1].psi);
                if (br < 0.5) {
                    atomic_max_pos(&maxv[2 + y], x + (a - 0.5) / (a - br));
                    rowbits |= 4u;
                }
            }
        }
        // freezing front on the centre column (lowest f_s = 1/2 crossing)
        if (x == nx / 2) {
            const double fa = double(m.fs);
            if (y == 0 && fa >= 0.5) atomicOr(bad + 1, 1u);
            if (fa >= 0.5) {
                if (y == ny - 1) {
                    atomic_min_pos(&minv[0], (double)ny);
                } else {
                    const double fb = double(fs[ey + 1][ex]);
                    if (fb < 0.5) atomic_min_pos(&minv[0], y + (fa - 0.5) / (fa - fb) + 0.5);
                }
            }
        }
    }
};

// One step that also reduces the observables of the
// state it starts from.  io, rng, cur as for k_step; `ws` carries this
// grid's block and group counts.
template <typename S, typename T, typename A, int BY, int PH>
__global__ void __launch_bounds__(32 * BY, step_min_blocks<S, T, BY>())
    k_step_obs(StepIO<S, T, A> io, Consts<T> c, Shift sh, ObsScratch ws, Scalars sc) {
    __shared__ TileSmem<T, BY> sm;
    __shared__ T s_fs[BY + 2][34], s_Tm[BY + 2][34];
    extern __shared__ __align__(16) unsigned char dsm_stash[];     // NPOP x BY x 32 values
    T(*stash)[BY][32] = reinterpret_cast<T(*)[BY][32]>(dsm_stash);
    // as k_step: FP32 and FP64 wait for k_halo inside step_tile
    constexpr bool EARLY = std::is_same<S, T>::value && std::is_same<typename FStore<S>::type, S>::value;
    if constexpr (!EARLY) grid_dep_wait();
    grid_dep_release();
    load_counters(io, PH);
    advance_counters(io, PH, blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0);
    StepObs<T, BY> ob;
    ob.fs = s_fs;
    ob.Tm = s_Tm;
    ob.maxv = ws.maxv;
    ob.minv = ws.minv;
    ob.bad = ws.bad;
#pragma unroll
    for (int j = 0; j < OBS_NSUM; j++) ob.v[j] = typename StepObs<T, BY>::R(0);
    ob.rowbits = 0u;
    step_tile<S, T, A, BY, PH, true, StepObs<T, BY>, EARLY>(io, c, sh, sm, stash, blockIdx.x * 32, blockIdx.y * BY,
                                                            &ob);
    obs_block_finish<32 * BY>(ws, ob.v, ob.rowbits, (int)(blockIdx.y * BY + threadIdx.y), io.ny);
}

// Local substrate heat flux (R24), one thread per column, in the step's
// arithmetic: -k(x,0) (4 T(x,1) - T(x,2) - 3 T(x,0)) / 2.  Needs ny >= 3.
template <typename S, typename T, typename A>
__global__ void k_heat_flux(DevState s, int cur, int lcur, Consts<T> c, Shift sh, double *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= s.nx) return;
    const PopView<S> pv = PopView<S>::at(s, cur, lcur);
    const A *aux = reinterpret_cast<const A *>(cur ? s.aux[1] : s.aux[0]);
    Macro<T> m0, m1, m2;
    cell_macros_t<S, T, A>(pv, aux, x, 0, c, sh, m0);
    cell_macros_t<S, T, A>(pv, aux, x, 1, c, sh, m1);
    cell_macros_t<S, T, A>(pv, aux, x, 2, c, sh, m2);
    const T k0 = chi(m0.fs, m0.psi, c.kth);
    out[x] = double(-k0 * (T(4) * m1.T_ - m2.T_ - T(3) * m0.T_) / T(2));
}

// ---------------------------------------------------------------------------
// Field access for tests and hand-over: stored planes <-> host doubles.
// ---------------------------------------------------------------------------
template <typename S, typename T, typename A>
__global__ void k_get(DevState s, int cur, int lcur, int field, Consts<double> c, Shift sh, double *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= s.nx || y >= s.ny) return;
    const long long P = s.plane, k = (long long)y * s.pitch + x;
    const long long N = (long long)s.nx * s.ny, o = (long long)y * s.nx + x;
    const PopView<S> pv = PopView<S>::at(s, cur, lcur);
    const A *aux = reinterpret_cast<const A *>(cur ? s.aux[1] : s.aux[0]);
    Refs<T> rf;
    Consts<T> ct;
    ct.phi_bot = T(c.phi_bot);
    ct.phi_top = T(c.phi_top);
    make_refs<S, T>(rf, sh, ct, y, s.ny);
    if (field == LBM_FIELD_F) {
#pragma unroll
        for (int i = 0; i < 9; i++)
            out[i * N + o] =
                double(Pol<typename FStore<S>::type, T>::ld(pv.pl.f + pv.o9(i, x, y), rf.f[i], 1.0f / sh.f_scale));
    } else if (field == LBM_FIELD_H) {
#pragma unroll
        for (int i = 0; i < 9; i++)
            out[i * N + o] = double(Pol<S, T>::ld(pv.pl.h + pv.o9(i, x, y), T(0), 1.0f / sh.h_scale));
    } else if (field == LBM_FIELD_G) {
#pragma unroll
        for (int i = 0; i < 9; i++)
            out[i * N + o] = double(Pol<S, T>::ld(pv.pl.g + pv.o9(i, x, y), rf.g[i], 1.0f / sh.g_scale));
    } else if (field == LBM_FIELD_L) {
#pragma unroll
        for (int i = 0; i < 5; i++)
            out[i * N + o] = double(Pol<S, T>::ld(pv.pl.l + pv.o5(i, x, y), rf.l[i], 1.0f / sh.l_scale));
    } else if (field >= LBM_FIELD_FS_PREV && field <= LBM_FIELD_S) {
        out[o] = double(aux[(field - LBM_FIELD_FS_PREV) * P + k]);
    } else if (field == LBM_FIELD_SIGMA) {
        out[o] = double(reinterpret_cast<const A *>(s.sigma)[k]);
    } else {
        Macro<double> m;
        obs_macros<S, T, A>(pv, aux, x, y, c, sh, m);
        out[o] = field == LBM_FIELD_PSI ? m.psi
               : field == LBM_FIELD_FSOLID ? m.fs
               : field == LBM_FIELD_T ? m.T_
               : field == LBM_FIELD_PHI ? m.phi
               : m.H;
    }
}

// Pre-solve residual.  The populations are streamed in place, so the change
// of phi over one sweep is measured against a snapshot: k_phi_snap stores phi
// of the current state (arithmetic type, in a spare auxiliary plane), the
// sweep runs, and k_phi_change takes the largest |phi - snapshot| as the bit
// pattern of a non-negative double (one atomic maximum per warp).
template <typename S, typename T, typename A>
__device__ __forceinline__ T phi_of(const PopView<S> &v, const Consts<double> &c, const Shift &sh, int x, int y) {
    Refs<T> rf;
    Consts<T> ct;
    ct.phi_bot = T(c.phi_bot);
    ct.phi_top = T(c.phi_top);
    make_refs<S, T>(rf, sh, ct, y, v.ny);
    T a = T(0);
#pragma unroll
    for (int i = 1; i < 5; i++) a += Pol<S, T>::ld(v.pl.l + v.o5(i, x, y), rf.l[i], 1.0f / sh.l_scale);
    return a / (T(1) - w5<T>(0));
}

template <typename S, typename T, typename A>
__global__ void k_phi_snap(DevState s, int lcur, Consts<double> c, Shift sh, A *snap) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= s.nx || y >= s.ny) return;
    snap[(long long)y * s.pitch + x] = A(phi_of<S, T, A>(PopView<S>::at(s, 0, lcur), c, sh, x, y));
}

template <typename S, typename T, typename A>
__global__ void k_phi_change(DevState s, int lcur, Consts<double> c, Shift sh, const A *snap, unsigned long long *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double d = 0.0;
    if (x < s.nx && y < s.ny) {
        const T now = phi_of<S, T, A>(PopView<S>::at(s, 0, lcur), c, sh, x, y);
        d = fabs(double(now) - double(T(snap[(long long)y * s.pitch + x])));
        if (!(d == d)) d = __longlong_as_double(0x7ff0000000000000ll);    // NaN counts as infinite
    }
    unsigned long long v = (unsigned long long)__double_as_longlong(d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// Natural-layout population planes (a snapshot body: f, h, g, l planes of
// `pitch` x ny elements) written into the in-place layout of phases
// (cur, lcur): each value goes to the slot that holds it there; raw
// elements, no conversion (the half-storage references depend on the
// direction and the reading cell only, the same in both layouts).
template <typename S, typename T, typename A>
__global__ void k_place(DevState s, int cur, int lcur, const void *src) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= s.nx || y >= s.ny) return;
    using F = typename FStore<S>::type;
    const PopView<S> pv = PopView<S>::at(s, cur, lcur);
    const Planes<S> in = Planes<S>::at(src, s.plane);
    const uint32_t P = (uint32_t)s.plane, k = (uint32_t)y * (uint32_t)s.pitch + (uint32_t)x;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const uint32_t o = pv.o9(i, x, y);
        pv.pl.f[o] = static_cast<const F *>(in.f)[i * P + k];
        pv.pl.h[o] = in.h[i * P + k];
        pv.pl.g[o] = in.g[i * P + k];
    }
#pragma unroll
    for (int i = 0; i < 5; i++) pv.pl.l[pv.o5(i, x, y)] = in.l[i * P + k];
}

template <typename S, typename T, typename A>
__global__ void k_set(DevState s, int cur, int lcur, int field, Consts<T> c, Shift sh, const double *in) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= s.nx || y >= s.ny) return;
    const long long P = s.plane, k = (long long)y * s.pitch + x;
    const long long N = (long long)s.nx * s.ny, o = (long long)y * s.nx + x;
    const PopView<S> pv = PopView<S>::at(s, cur, lcur);
    A *aux = reinterpret_cast<A *>(cur ? s.aux[1] : s.aux[0]);
    Refs<T> rf;
    make_refs<S, T>(rf, sh, c, y, s.ny);
    // each value goes to the slot that holds it in the current layout
    if (field == LBM_FIELD_F) {
#pragma unroll
        for (int i = 0; i < 9; i++)
            Pol<typename FStore<S>::type, T>::st(pv.pl.f + pv.o9(i, x, y), T(in[i * N + o]), rf.f[i], sh.f_scale);
    } else if (field == LBM_FIELD_H) {
#pragma unroll
        for (int i = 0; i < 9; i++) Pol<S, T>::st(pv.pl.h + pv.o9(i, x, y), T(in[i * N + o]), T(0), sh.h_scale);
    } else if (field == LBM_FIELD_G) {
#pragma unroll
        for (int i = 0; i < 9; i++) Pol<S, T>::st(pv.pl.g + pv.o9(i, x, y), T(in[i * N + o]), rf.g[i], sh.g_scale);
    } else if (field == LBM_FIELD_L) {
#pragma unroll
        for (int i = 0; i < 5; i++) Pol<S, T>::st(pv.pl.l + pv.o5(i, x, y), T(in[i * N + o]), rf.l[i], sh.l_scale);
    } else if (field >= LBM_FIELD_FS_PREV && field <= LBM_FIELD_S) {
        aux[(field - LBM_FIELD_FS_PREV) * P + k] = A(in[o]);
    } else if (field == LBM_FIELD_SIGMA) {
        reinterpret_cast<A *>(s.sigma)[k] = A(in[o]);
    }
}

}  // namespace lbm
