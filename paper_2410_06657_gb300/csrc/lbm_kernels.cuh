// Fused sm_103a kernels of the phase-field LB electrofreezing step
// (arXiv 2410.06657, Secs. 2-3 and Algorithm 1), templated on
//   S  storage type of the populations (double, float, __half),
//   T  arithmetic type (double or float),
//   A  type of the auxiliary per-cell fields (double or float).
// Included once by each precision's translation unit.
//
// Memory layout (all structure-of-arrays, x fastest, rows padded to `pitch`):
//   pop     : ONE copy of 32 planes  f_0..8 | h_0..8 | g_0..8 | l_0..4 (half
//             storage: the f planes in float, the others in half), streamed
//             in place with the AA pattern (below); f, h, g share a layout
//             phase that flips every step, l keeps its own because the extra
//             potential sweeps flip it alone
//   aux[b]  : 7 planes   f_s, mdot, rho C_p T mdot, psi u_x, psi u_y, p, S
//             of the previous step (read by the next step's stencils, so the
//             step reads copy b and writes copy 1-b)
//   sigma   : conductivity at time n for the extra potential sweeps
//   halo    : (psi, f_s, phi) of every tile-edge cell at the current time
//             level, one 16-byte (FP64: 32-byte) record per cell
//
// One step is two launches over the same 32 x BY tiles.  k_halo computes
// the local macroscopic fields of every tile-edge cell (the cells another
// tile's one-cell ring holds) into the halo records.  k_step then computes
// the local macroscopic fields of its own cells into shared memory and takes
// its ring from the records (rho and eps follow from (psi, f_s) by the
// property law), applies the radius-1 stencils, forces, flow macros, the
// four collisions and writes the post-collision populations back into the
// slots the cell read, with the wall rules.  The launch boundary orders
// every record store before every population is overwritten, so no block
// ever reads a value another block of the same launch writes.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "lbm_internal.h"
#include "philox.h"

namespace lbm {

// D2Q9 (Sec. 3.1): rest; E, N, W, S; NE, NW, SW, SE.
__device__ constexpr int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ constexpr int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
__device__ constexpr int PAIR9[4] = {1, 2, 5, 6};   // one direction of each opposite pair
// D2Q5 (Sec. 3.4): rest; E, N, W, S.
__device__ constexpr int CX5[5] = {0, 1, 0, -1, 0};
__device__ constexpr int CY5[5] = {0, 0, 1, 0, -1};
__device__ constexpr int OPP5[5] = {0, 3, 4, 1, 2};

template <typename T>
__device__ __forceinline__ constexpr T w9(int i) {
    return i == 0 ? T(4.0 / 9.0) : (i < 5 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}
template <typename T>
__device__ __forceinline__ constexpr T w5(int i) {
    return i == 0 ? T(1.0 / 3.0) : T(1.0 / 6.0);
}
template <typename T>
__device__ __forceinline__ constexpr T cs2() { return T(1.0 / 3.0); }

// ---------------------------------------------------------------------------
// Storage policies: how a population of arithmetic type T is kept in S.
// ---------------------------------------------------------------------------
template <typename S, typename T>
struct Pol {
    static constexpr bool shifted = false;
    __device__ static __forceinline__ T ld(const S *p, T, float) { return T(*p); }
    __device__ static __forceinline__ void st(S *p, T v, T, float) { *p = S(v); }
    __device__ static __forceinline__ void st_sr(S *p, T v, T, float, uint32_t) { *p = S(v); }
};

// Stochastic rounding of a float to half: rounds away from zero with
// probability equal to the distance from the value truncated towards zero,
// in units of the half spacing, so the stored value is unbiased.  r13 holds
// 13 uniform random bits (the number of mantissa bits a float has beyond a
// half's).  The conversion is the PTX cvt with stochastic rounding (.rs),
// which takes the random bits from the caller: for a normal half it adds
// them to the 13 mantissa bits the half drops and truncates; in the
// subnormal half range (spacing 2^-24) the value moves by r13 * 2^-37
// towards larger magnitude before truncation; .satfinite keeps a value
// beyond the half range at the largest finite half, as truncation does.
// The f16x2 form converts two values at once, its second operand with bits
// 0-12 of the random word; one value goes in that slot.
__device__ __forceinline__ __half half_sr(float v, uint32_t r13) {
    uint32_t d;
    asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(0.0f), "f"(v), "r"(r13));
    return __ushort_as_half((unsigned short)(d & 0xffffu));
}
template <>
struct Pol<__half, float> {
    static constexpr bool shifted = true;
    __device__ static __forceinline__ float ld(const __half *p, float ref, float inv_scale) {
        return __fmaf_rn(__half2float(*p), inv_scale, ref);    // one rounding in every context
    }
    __device__ static __forceinline__ void st(__half *p, float v, float ref, float scale) {
        *p = __float2half_rn((v - ref) * scale);
    }
    __device__ static __forceinline__ void st_sr(__half *p, float v, float ref, float scale, uint32_t r13) {
        *p = half_sr((v - ref) * scale, r13);
    }
};

// Random bits of the stochastic rounding: one Philox block per cell, step
// and population system (counter), under a fixed key.  The enthalpy and
// potential populations are rounded stochastically; the flow populations
// change by more than half a spacing per step and are rounded to nearest.
constexpr uint32_t SR_KEY0 = 0x24100665u, SR_KEY1 = 0x0F16A5EDu;
__device__ __forceinline__ void sr_block(uint32_t w[4], long long k, uint32_t step, uint32_t sys) {
    w[0] = (uint32_t)k;
    w[1] = step;
    w[2] = sys;
    w[3] = 0u;
    philox4x32_10(w, SR_KEY0, SR_KEY1);
}

// Population planes of one buffer copy: f (9 planes of type F), then h (9),
// g (9) and l (5) of the storage type S.  Half storage keeps f in single
// precision: with f in half, the rounding noise on psi in the cold gas
// (where f is largest after the shift) becomes spurious solid through
// f_s = psi (1 - f_l) (negative excursions count as no solid, positive ones
// as solid), and the freezing time came out about 1 % early.
template <typename S> struct FStore { using type = S; };
template <> struct FStore<__half> { using type = float; };

template <typename S>
struct Planes {
    using F = typename FStore<S>::type;
    F *f;
    S *h, *g, *l;
    __host__ __device__ static Planes at(const void *base, long long P) {
        Planes v;
        char *b = const_cast<char *>(reinterpret_cast<const char *>(base));
        v.f = reinterpret_cast<F *>(b);
        v.h = reinterpret_cast<S *>(b + 9 * P * (long long)sizeof(F));
        v.g = v.h + 9 * P;
        v.l = v.h + 18 * P;
        return v;
    }
};

// Separately rounded product, sum and difference: the compiler never fuses
// these into an FMA, so a value built from them has the same bits wherever
// it is evaluated (a tile-edge cell's macros are computed by the halo kernel
// for its neighbour tiles and again by the step for the cell itself).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Per-cell reference values of the weight-shifted half storage.
template <typename T>
struct Refs {
    T f[9], g[9], l[5];
};

template <typename S, typename T>
__device__ __forceinline__ void make_refs(Refs<T> &r, const Shift &sh, const Consts<T> &c, int y,
                                          int ny) {
    if constexpr (Pol<S, T>::shifted) {
#pragma unroll
        for (int i = 0; i < 9; i++) {
            r.f[i] = mul_rn(w9<T>(i), T(sh.f_ref));
            r.g[i] = (i == 0) ? T(sh.g0_ref) : mul_rn(w9<T>(i), T(sh.g_ref));
        }
        // linear potential between the electrodes
        T phil = add_rn(c.phi_bot, mul_rn(sub_rn(c.phi_top, c.phi_bot), T(y) + T(0.5)) / T(ny));
#pragma unroll
        for (int i = 0; i < 5; i++) r.l[i] = mul_rn((i == 0) ? w5<T>(0) - T(1) : w5<T>(i), phil);
    }
}

// ---------------------------------------------------------------------------
// Pointwise physics (shared by the step, observables and field kernels).
// ---------------------------------------------------------------------------

// Eq. (Computed): three-phase property law, evaluated left to right.
template <typename T>
__device__ __forceinline__ T chi(T fs, T psi, const T v[3]) {
    const T ls = sub_rn(T(1), fs);
    const T a = mul_rn(fs, v[0]);
    const T b = mul_rn(mul_rn(ls, psi), v[1]);
    const T d = mul_rn(mul_rn(ls, sub_rn(T(1), psi)), v[2]);
    return add_rn(add_rn(a, b), d);
}

// Eq. (Hfl) with H_s = C_p T_m, latent heat carried by the liquid part
// (L_eff = psi L): liquid fraction and temperature from total enthalpy.
template <typename T>
__device__ __forceinline__ void enthalpy_inversion(T H, T psi, T cp, T Tm, T L, T &fl, T &Tt) {
    T Hs = mul_rn(cp, Tm);
    T Leff = mul_rn(psi, L);
    T Hl = add_rn(Hs, Leff);
    if (H < Hs)
        Tt = H / cp;
    else if (H <= Hl)
        Tt = Tm;
    else
        Tt = add_rn(Tm, sub_rn(H, Hl) / cp);
    if (Leff < T(1e-12)) {
        fl = T(1);
    } else {
        T r = sub_rn(H, Hs) / Leff;
        fl = r < T(0) ? T(0) : (r > T(1) ? T(1) : r);
    }
}

template <typename T>
struct Macro {
    T psi, H, T_, fs, rho, eps, phi;
};

// Local macroscopic quantities from the populations at time n
// (psi and H use the previous step's mdot and rho C_p T mdot).
template <typename T>
__device__ __forceinline__ void local_macros(const T f[9], const T g[9], T l1234, T fs_prev,
                                             T mdot_prev, T Q_prev, const Consts<T> &c,
                                             Macro<T> &m) {
    T sf = T(0);
#pragma unroll
    for (int i = 0; i < 9; i++) sf += f[i];
    m.psi = sf / sub_rn(T(1), mul_rn(T(0.5), mdot_prev));  // Eq. (Computed_psi)
    T sg = T(0);
#pragma unroll
    for (int i = 0; i < 9; i++) sg += g[i];
    m.H = add_rn(sg, mul_rn(T(0.5), Q_prev));              // Sec. 3.3
    T cp_lev = chi(fs_prev, m.psi, c.cp);
    T fl;
    enthalpy_inversion(m.H, m.psi, cp_lev, c.T_m, c.L, fl, m.T_);
    m.fs = mul_rn(m.psi, sub_rn(T(1), fl));
    m.rho = chi(m.fs, m.psi, c.rho);
    m.eps = chi(m.fs, m.psi, c.eps);
    m.phi = l1234 / (T(1) - w5<T>(0));                    // Eq. (Computed_phi)
}

// c . (a, b) for a lattice vector with components in {-1, 0, 1}.  Terms
// with a zero component are skipped and signs are applied exactly, so the
// result has the bits of cx * a + cy * b evaluated in that order (adding a
// signed zero or multiplying by +-1 is exact) without the zero products.
template <typename T>
__device__ __forceinline__ T cdot(int cx, int cy, T a, T b) {
    T r = cx > 0 ? a : (cx < 0 ? -a : T(0));
    if (cy > 0) r = cx != 0 ? r + b : b;
    else if (cy < 0) r = cx != 0 ? r - b : -b;
    return r;
}

// Isotropic stencils (Eqs. eqtidi1-2) on the nine values v[i] = z(x + c_i):
// the sums over i = 1..8 of w_i c_i v_i and 2 w_i (v_i - v_0), divided by
// c_s^2, in the order of i with the zero terms of the gradient left out.
// RED (single-precision storage only): an algebraically equal form with
// opposite neighbours differenced first, the diagonal differences shared by
// both components and 1/c_s^2 = 3 folded into the weights.
template <typename S>
constexpr bool reduced_stencils() { return std::is_same<S, float>::value; }

template <typename T, bool RED = false>
__device__ __forceinline__ void grad_v(const T v[9], T &gx, T &gy) {
    if constexpr (RED && sizeof(T) == 4) {
        const T d13 = v[1] - v[3], d24 = v[2] - v[4];
        const T d57 = v[5] - v[7], d86 = v[8] - v[6];
        gx = T(1.0 / 3.0) * d13 + T(1.0 / 12.0) * (d57 + d86);
        gy = T(1.0 / 3.0) * d24 + T(1.0 / 12.0) * (d57 - d86);
        return;
    }
    const T wa = T(1.0 / 9.0), wd = T(1.0 / 36.0);
    T sx = wa * v[1];
    sx = sx - wa * v[3];
    sx = sx + wd * v[5];
    sx = sx - wd * v[6];
    sx = sx - wd * v[7];
    sx = sx + wd * v[8];
    T sy = wa * v[2];
    sy = sy - wa * v[4];
    sy = sy + wd * v[5];
    sy = sy + wd * v[6];
    sy = sy - wd * v[7];
    sy = sy - wd * v[8];
    gx = sx / cs2<T>();
    gy = sy / cs2<T>();
}
template <typename T, bool RED = false>
__device__ __forceinline__ T lap_v(const T v[9]) {
    if constexpr (RED && sizeof(T) == 4) {
        // 6 (w_a sum of the axis neighbours + w_d sum of the diagonal ones) - 6 (4 w_a + 4 w_d) v_0
        const T sa = (v[1] + v[3]) + (v[2] + v[4]);
        const T sd = (v[5] + v[7]) + (v[6] + v[8]);
        return T(2.0 / 3.0) * sa + (T(1.0 / 6.0) * sd - T(10.0 / 3.0) * v[0]);
    }
    T acc = T(0);
#pragma unroll
    for (int i = 1; i < 9; i++) acc += T(2) * w9<T>(i) * (v[i] - v[0]);
    return acc / cs2<T>();
}

// The same stencils on a shared-memory tile, so a stencil evaluated by the
// observables kernel and by the step gives the same bits.
template <typename T, int W>
__device__ __forceinline__ void load9(const T (*z)[W], int ex, int ey, T v[9]) {
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = z[ey + CY[i]][ex + CX[i]];
}
template <typename T, int W, bool RED = false>
__device__ __forceinline__ void grad_s(const T (*z)[W], int ex, int ey, T &gx, T &gy) {
    T v[9];
    load9<T, W>(z, ex, ey, v);
    grad_v<T, RED>(v, gx, gy);
}
template <typename T, int W, bool RED = false>
__device__ __forceinline__ T lap_s(const T (*z)[W], int ex, int ey) {
    T v[9];
    load9<T, W>(z, ex, ey, v);
    return lap_v<T, RED>(v);
}

// s_i(u) of Sec. 3.2.
template <typename T>
__device__ __forceinline__ T s_i(int i, T ux, T uy) {
    T cu = cdot<T>(CX[i], CY[i], ux, uy);
    T uu = ux * ux + uy * uy;
    return w9<T>(i) * (cu / cs2<T>() + cu * cu / (T(2) * cs2<T>() * cs2<T>()) - uu / (T(2) * cs2<T>()));
}

template <typename T>
__device__ __forceinline__ int wrapx(int x, int nx) {
    return x < 0 ? x + nx : (x >= nx ? x - nx : x);
}

// Slot r of the one-cell ring around a 32 x BY tile, in extended-tile
// coordinates (row 0 and row BY+1 are 34 wide, columns 0 and 33 BY high).
template <int BY>
__device__ __forceinline__ void ring_slot(int r, int &ex, int &ey) {
    if (r < 34) {
        ex = r; ey = 0;
    } else if (r < 68) {
        ex = r - 34; ey = BY + 1;
    } else if (r < 68 + BY) {
        ex = 0; ey = r - 68 + 1;
    } else {
        ex = 33; ey = r - 68 - BY + 1;
    }
}


// ---------------------------------------------------------------------------
// In-place streaming: the AA pattern (Bailey, Myre, Walsh, Lilja and Saar,
// ICPP 2009).  One copy of the populations holds the state in one of two
// layouts, which alternate from step to step:
//   phase 0 (natural): population i of cell x sits in plane i at x;
//   phase 1 (swapped): population i of cell x sits in plane opp(i) at the
//     upstream cell x - c_i, or in plane i at x itself where x - c_i lies
//     beyond a wall (the previous step left the bounced-back value there).
// A step from phase 0 reads each cell's own slots and writes the
// post-collision population i into plane opp(i) of the same cell (already
// bounced back where x + c_i lies beyond a wall); a step from phase 1 reads
// through the swapped layout and pushes population i into plane i at
// x + c_i (into a wall: back into plane opp(i) at x).  Either way a cell
// writes exactly the slots it read and no other cell writes them, so the
// update is race-free in place.  x is periodic.  Half storage keeps the
// reference of (direction, row of the cell that will read the value), as
// the two-copy push did, so a slot's raw bits mean the same in both layouts.
// ---------------------------------------------------------------------------

// Offset (plane times P plus the cell offset) of the slot holding population
// i of cell (x, y) at the start of a step from phase ph, relative to the
// system's first plane; xm, xp are x - 1 and x + 1 wrapped.
template <int NQ>
__device__ __forceinline__ uint32_t aa_src(int ph, int i, uint32_t P, uint32_t pitch, int x, int y, int xm, int xp,
                                           int ny) {
    const int cx = NQ == 9 ? CX[i] : CX5[i], cy = NQ == 9 ? CY[i] : CY5[i];
    const int io = NQ == 9 ? OPP9[i] : OPP5[i];
    const uint32_t own = (uint32_t)i * P + (uint32_t)y * pitch + (uint32_t)x;
    if (ph == 0 || (cx == 0 && cy == 0)) return own;
    const int yu = y - cy;
    if (yu < 0 || yu >= ny) return own;
    const int xu = cx > 0 ? xm : (cx < 0 ? xp : x);
    return (uint32_t)io * P + (uint32_t)yu * pitch + (uint32_t)xu;
}

// Destination of cell (x, y)'s post-collision population i in a step from
// phase ph; `wall` tells whether it leaves through a wall, in which case the
// slot receives the bounced value (population opp(i) of the cell itself).
// EDGE false: the tile touches no wall row, so no direction leaves.
template <int NQ, bool EDGE>
__device__ __forceinline__ uint32_t aa_dst(int ph, int i, uint32_t P, uint32_t pitch, int x, int y, int xm, int xp,
                                           int ny, bool &wall) {
    const int cx = NQ == 9 ? CX[i] : CX5[i], cy = NQ == 9 ? CY[i] : CY5[i];
    const int io = NQ == 9 ? OPP9[i] : OPP5[i];
    const int yt = y + cy;
    wall = EDGE && (yt < 0 || yt >= ny);
    if (ph == 0 || wall) return (uint32_t)io * P + (uint32_t)y * pitch + (uint32_t)x;
    const int xt = cx > 0 ? xp : (cx < 0 ? xm : x);
    return (uint32_t)i * P + (uint32_t)yt * pitch + (uint32_t)xt;
}

// ---------------------------------------------------------------------------
// Halo records: (psi, f_s, phi) of a tile-edge cell at time n, written by
// k_halo and read by the step kernel of the same step.  FP32 packs them in
// one 16-byte vector, FP64 in two.
// ---------------------------------------------------------------------------
template <typename T>
struct alignas(4 * sizeof(T)) HaloRec {
    T psi, fs, phi, pad;
};

__device__ __forceinline__ void st_halo(HaloRec<float> *p, float psi, float fs, float phi) {
    *reinterpret_cast<float4 *>(p) = make_float4(psi, fs, phi, 0.0f);
}
__device__ __forceinline__ void st_halo(HaloRec<double> *p, double psi, double fs, double phi) {
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(psi, fs);
    q[1] = make_double2(phi, 0.0);
}
// Loaded from L2: the records change every step.
__device__ __forceinline__ void ld_halo(const HaloRec<float> *p, float &psi, float &fs, float &phi) {
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    psi = v.x;
    fs = v.y;
    phi = v.z;
}
__device__ __forceinline__ void ld_halo(const HaloRec<double> *p, double &psi, double &fs, double &phi) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 a = __ldcg(q), b = __ldcg(q + 1);
    psi = a.x;
    fs = a.y;
    phi = b.x;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may be scheduled while the kernel before it in the stream
// drains; grid_dep_wait() returns once that kernel has completed and its
// stores are visible, and grid_dep_release() lets the next such kernel be
// scheduled.  Every kernel of a step waits before its first global load, so
// only the launch latency overlaps.  Both are no-ops in a kernel launched
// without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


// ---------------------------------------------------------------------------
// The fused step for one 32 x BY tile.
// ---------------------------------------------------------------------------
template <typename T, int BY>
struct TileSmem {
    // per extended-tile cell, packed so a stencil reads each neighbour with
    // one vector load: (psi, rho, eps, phi) and (p, S)
    struct alignas(4 * sizeof(T)) Quad { T psi, rho, eps, phi; };
    struct alignas(2 * sizeof(T)) Pair { T p, S; };
    Quad q[BY + 2][34];
    Pair ps[BY + 2][34];
};

template <typename S, typename T, typename A>
struct StepIO {
    using F = typename FStore<S>::type;
    F *f;                    // population planes (one copy, streamed in place)
    S *h, *g, *l;
    const A *aux_in;
    A *aux_out;
    A *sigma;
    HaloRec<T> *hm;          // halo records of the tile-edge cells
    unsigned int *rng;       // [2] stochastic-rounding counters (half storage) or null
    int nx, ny, pitch, write_sigma, lph;
    long long plane;
    uint32_t sr_step;        // this step's stochastic-rounding counter (half storage)
};

// The step's pointers and sizes for the parities (cur, lcur): cur is the
// layout phase of f, h, g and selects the auxiliary copy, lcur the phase of
// l.  The host resolves them for the single-instance kernels.
template <typename S, typename T, typename A>
__host__ __device__ __forceinline__ StepIO<S, T, A> step_io(const DevState &s, int cur, int lcur, int write_sigma) {
    StepIO<S, T, A> io;
    const Planes<S> pl = Planes<S>::at(s.pop, s.plane);
    io.f = pl.f;
    io.h = pl.h;
    io.g = pl.g;
    io.l = pl.l;
    // select rather than index the parameter arrays (a dynamic index would
    // copy them to local memory)
    io.aux_in = reinterpret_cast<const A *>(cur ? s.aux[1] : s.aux[0]);
    io.aux_out = reinterpret_cast<A *>(cur ? s.aux[0] : s.aux[1]);
    io.sigma = reinterpret_cast<A *>(s.sigma);
    io.hm = reinterpret_cast<HaloRec<T> *>(s.halo);
    io.rng = s.rng;
    io.sr_step = 0u;
    io.nx = s.nx;
    io.ny = s.ny;
    io.pitch = s.pitch;
    io.write_sigma = write_sigma;
    io.lph = lcur;
    io.plane = s.plane;
    return io;
}

// The step's counters live in device memory (graph replays advance them):
// counter[cur] is this step's, and one thread writes counter[cur ^ 1] for
// the next step (parities flipped), which no thread of this step reads.
template <typename S, typename T, typename A>
__device__ __forceinline__ void load_counters(StepIO<S, T, A> &io, int cur) {
    if constexpr (Pol<S, T>::shifted) {
        if (io.rng) io.sr_step = io.rng[cur];
    }
}
template <typename S, typename T, typename A>
__device__ __forceinline__ void advance_counters(const StepIO<S, T, A> &io, int cur, bool leader) {
    if (!leader) return;
    if constexpr (Pol<S, T>::shifted) {
        if (io.rng) io.rng[cur ^ 1] = io.sr_step + 1u;
    }
}

// Observation hooks of a step: a plain step observes nothing.  A step that
// also reduces the observables of the state it starts from passes an
// observer (lbm_observe.cuh) that keeps the macros it needs from phase 1 and
// adds every own cell's terms after the cell's push.
struct NoObs {};

// The stored values one cell's macros need, in the arithmetic type T.
template <typename T>
struct CellLoad {
    T f[9], g[9], l1234, fs_prev, mdot_prev, Q_prev;
};

// Loads of cell (x, y)'s stored values for its macros, through the layout
// of phases (PH, io.lph), and its previous-step (p, S).
template <typename S, typename T, typename A, int PH>
__device__ __forceinline__ void load_cell_aa(const StepIO<S, T, A> &io, const Consts<T> &c, const Shift &sh, int x,
                                             int y, CellLoad<T> &o, T &pv, T &Sv) {
    const uint32_t P = (uint32_t)io.plane, pitch = (uint32_t)io.pitch;
    const int xm = x == 0 ? io.nx - 1 : x - 1, xp = x == io.nx - 1 ? 0 : x + 1;
    const uint32_t k = (uint32_t)y * pitch + (uint32_t)x;
    Refs<T> rf;
    make_refs<S, T>(rf, sh, c, y, io.ny);
    const float fi = 1.0f / sh.f_scale, gi = 1.0f / sh.g_scale, li = 1.0f / sh.l_scale;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const uint32_t o9 = aa_src<9>(PH, i, P, pitch, x, y, xm, xp, io.ny);
        o.f[i] = Pol<typename FStore<S>::type, T>::ld(io.f + o9, rf.f[i], fi);
        o.g[i] = Pol<S, T>::ld(io.g + o9, rf.g[i], gi);
    }
    o.l1234 = T(0);
#pragma unroll
    for (int i = 1; i < 5; i++)
        o.l1234 += Pol<S, T>::ld(io.l + aa_src<5>(io.lph, i, P, pitch, x, y, xm, xp, io.ny), rf.l[i], li);
    o.fs_prev = T(io.aux_in[AUX_FS * P + k]);
    o.mdot_prev = T(io.aux_in[AUX_MDOT * P + k]);
    o.Q_prev = T(io.aux_in[AUX_Q * P + k]);
    pv = T(io.aux_in[AUX_P * P + k]);
    Sv = T(io.aux_in[AUX_S * P + k]);
}

// The halo record of a tile-edge cell: its time-n macros from its own
// populations, exactly as the cell's owner computes them.
template <typename S, typename T, typename A, int PH>
__device__ __forceinline__ void halo_cell(const StepIO<S, T, A> &io, const Consts<T> &c, const Shift &sh, int x,
                                          int y) {
    CellLoad<T> ld;
    T pv, Sv;
    load_cell_aa<S, T, A, PH>(io, c, sh, x, y, ld, pv, Sv);
    Macro<T> m;
    local_macros<T>(ld.f, ld.g, ld.l1234, ld.fs_prev, ld.mdot_prev, ld.Q_prev, c, m);
    st_halo(io.hm + (size_t)y * io.pitch + x, m.psi, m.fs, m.phi);
}

// The ring cell (x, y) of a tile, loaded from its halo record and its
// previous-step (p, S).
template <typename T>
struct RingLoad {
    T psi, fs, phi, p, S;
};
template <typename S, typename T, typename A>
__device__ __forceinline__ void ring_load(const StepIO<S, T, A> &io, int x, int y, RingLoad<T> &r) {
    const uint32_t P = (uint32_t)io.plane;
    const uint32_t k = (uint32_t)y * (uint32_t)io.pitch + (uint32_t)x;
    ld_halo(io.hm + k, r.psi, r.fs, r.phi);
    r.p = T(io.aux_in[AUX_P * P + k]);
    r.S = T(io.aux_in[AUX_S * P + k]);
}
// ... into the extended tile slot (ex, ey): rho and eps by the property law
// from (psi, f_s), as local_macros evaluates them.
template <typename T, int BY, typename OB>
__device__ __forceinline__ void ring_to_smem(const Consts<T> &c, const RingLoad<T> &r, TileSmem<T, BY> &sm, int ex,
                                             int ey, OB *ob) {
    Macro<T> m;
    m.psi = r.psi;
    m.fs = r.fs;
    m.phi = r.phi;
    m.rho = chi(m.fs, m.psi, c.rho);
    m.eps = chi(m.fs, m.psi, c.eps);
    m.H = T(0);
    m.T_ = T(0);
    sm.q[ey][ex] = {m.psi, m.rho, m.eps, m.phi};
    sm.ps[ey][ex] = {r.p, r.S};
    if constexpr (!std::is_same<OB, NoObs>::value) ob->macro(ey, ex, m);
}

// Asynchronous global -> shared copy of one 4- or 8-byte element.
template <typename V>
__device__ __forceinline__ void cp_async_elem(V *dst_smem, const V *src) {
    static_assert(sizeof(V) == 4 || sizeof(V) == 8, "cp.async element size");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    if constexpr (sizeof(V) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Warp-cooperative 16-byte copies of one full tile row (32 cells starting at
// offset k0, a multiple of 32 elements, so every chunk is 16-byte aligned)
// of the population planes into the stash: each warp instruction moves
// 32 / CR planes, lane tx copies chunk tx % CR of plane j * (32 / CR) +
// tx / CR.  Planes 0-26 (f, h, g) lie contiguously from pin, planes 27-31
// (l) from lin; with l_all false only planes 0-27 are copied (the rest
// population l_0 is in place in either layout, l_1..4 are then gathered by
// the caller).  A quarter (FP32) or half (FP64) of the instructions of one
// copy per element.
// CG: the copies bypass L1 (cp.async.cg).
template <typename T, int BY, bool CG = false>
__device__ __forceinline__ void stash_row_async(T (*stash)[BY][32], int ty, int tx, const T *pin,
                                                const T *lin, uint32_t P, uint32_t k0, bool l_all) {
    constexpr int CR = 32 * int(sizeof(T)) / 16;    // 16-byte chunks per row
    constexpr int PPJ = 32 / CR;                    // planes per instruction
    constexpr int EPC = 16 / int(sizeof(T));        // elements per chunk
    static_assert(28 % PPJ == 0, "planes 28-31 start an instruction");
    const int part = tx % CR, sub = tx / CR;
#pragma unroll
    for (int j = 0; j < CR; j++) {
        if (j * PPJ >= 28 && !l_all) break;
        const int q = j * PPJ + sub;
        const T *src;
        if (j * PPJ + PPJ <= 27)
            src = pin + ((uint32_t)q * P + k0);
        else if (j * PPJ >= 27)
            src = lin + ((uint32_t)(q - 27) * P + k0);
        else
            src = q < 27 ? pin + ((uint32_t)q * P + k0) : lin + ((uint32_t)(q - 27) * P + k0);
        const unsigned d = (unsigned)__cvta_generic_to_shared(&stash[q][ty][part * EPC]);
        if constexpr (CG)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + part * EPC) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + part * EPC) : "memory");
    }
}

// Population sources for step_cell.
template <typename T, int BY>
struct StashPops {            // own cell's populations stashed in shared memory
    const T (*q)[BY][32];
    int ty, tx;
    __device__ __forceinline__ T f(int i) const { return q[i][ty][tx]; }
    __device__ __forceinline__ T h(int i) const { return q[9 + i][ty][tx]; }
    __device__ __forceinline__ T g(int i) const { return q[18 + i][ty][tx]; }
    __device__ __forceinline__ T l(int i) const { return q[27 + i][ty][tx]; }
};

// Wall ghost rows of the stencil tile (readings R17, R19): wetting ghost of
// psi at the bottom wall, neutral at the top, copies of rho, eps, p, S, and
// phi mirrored about the electrode potential.
template <typename T, int BY>
__device__ __forceinline__ void fill_ghosts(TileSmem<T, BY> &sm, const Consts<T> &c, int y0, int ny, int tid) {
    if (y0 == 0 && tid < 34) {              // bottom wall: wetting, copy, mirror
        const typename TileSmem<T, BY>::Quad a = sm.q[1][tid];
        const T z = a.psi;
        sm.q[0][tid] = {z + c.wet * z * (T(1) - z), a.rho, a.eps, T(2) * c.phi_bot - a.phi};
        sm.ps[0][tid] = sm.ps[1][tid];
    }
    const int et = ny - y0 + 1;              // ext row of y = ny, if inside the tile
    if (et >= 1 && et <= BY + 1 && tid >= 64 && tid < 98) {
        const int e = tid - 64;              // top wall: neutral wetting, copy, mirror
        const typename TileSmem<T, BY>::Quad a = sm.q[et - 1][e];
        sm.q[et][e] = {a.psi, a.rho, a.eps, T(2) * c.phi_top - a.phi};
        sm.ps[et][e] = sm.ps[et - 1][e];
    }
}

// The rest of the step for one own cell: stencils from the shared-memory tile, forces,
// flow macros, the four collisions and the write-back of the post-collision
// populations through the AA pattern from phase PH (l: io.lph).  PS
// supplies the cell's time-n populations (registers or shared memory).
// EDGE: the tile touches a wall row, so destinations may leave the lattice;
// interior tiles skip the per-direction wall tests.
template <typename S, typename T, typename A, int BY, bool EDGE, int PH, typename PopSrc, typename OB = NoObs>
__device__ __forceinline__ void step_cell(const StepIO<S, T, A> &io, const Consts<T> &c, const Shift &sh,
                                          const TileSmem<T, BY> &sm, const PopSrc &PS, int tx, int ty, int x,
                                          int y, const Macro<T> &m, T fs_prev, T pux_prev, T puy_prev,
                                          OB *ob = nullptr) {
    const int nx = io.nx, ny = io.ny;
    const uint32_t P = (uint32_t)io.plane;   // 32-bit offsets (checked at creation)
    const uint32_t pitch = (uint32_t)io.pitch;
    const uint32_t k = (uint32_t)y * pitch + (uint32_t)x;
    Refs<T> ro;                               // destination references (half storage)
    const int ex = tx + 1, ey = ty + 1;
    // ---- a2: stencils ----------------------------------------------------
    T gpsix, gpsiy, grhox, grhoy, gepsx, gepsy, gphix, gphiy, gpx, gpy, gSx, gSy, lpsi, lphi;
    {
        T vpsi[9], vrho[9], veps[9], vphi[9], vp[9], vS[9];
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const typename TileSmem<T, BY>::Quad a = sm.q[ey + CY[i]][ex + CX[i]];
            const typename TileSmem<T, BY>::Pair b = sm.ps[ey + CY[i]][ex + CX[i]];
            vpsi[i] = a.psi; vrho[i] = a.rho; veps[i] = a.eps; vphi[i] = a.phi;
            vp[i] = b.p; vS[i] = b.S;
        }
        constexpr bool RED = reduced_stencils<S>();
        grad_v<T, RED>(vpsi, gpsix, gpsiy);
        lpsi = lap_v<T, RED>(vpsi);
        grad_v<T, RED>(vrho, grhox, grhoy);
        grad_v<T, RED>(veps, gepsx, gepsy);
        grad_v<T, RED>(vphi, gphix, gphiy);
        lphi = lap_v<T, RED>(vphi);
        grad_v<T, RED>(vp, gpx, gpy);
        grad_v<T, RED>(vS, gSx, gSy);
    }

    // ---- a3: forces (Eq. Fs with the chemical potential of Sec. 2; Eq. Fe)
    const T ps = m.psi;
    const T muc = T(4) * c.beta * (ps - T(1)) * (ps - T(0)) * (ps - T(0.5)) - c.kappa * lpsi;
    const T Fsx = muc * gpsix, Fsy = muc * gpsiy;
    const T Ex = -gphix, Ey = -gphiy;
    const T qv = -(gepsx * gphix + gepsy * gphiy + m.eps * lphi);
    const T E2 = Ex * Ex + Ey * Ey;
    const T Fex = qv * Ex - T(0.5) * E2 * gepsx;
    const T Fey = qv * Ey - T(0.5) * E2 * gepsy;
    const T Fx = Fsx + Fex, Fy = Fsy + Fey;

    // ---- a4: flow macros (Sec. 3.2) ---------------------------------------
    // sum_i c_i h_i in the order of i (zero terms skipped)
    T jx = PS.h(1);
    jx = jx - PS.h(3);
    jx = jx + PS.h(5);
    jx = jx - PS.h(6);
    jx = jx - PS.h(7);
    jx = jx + PS.h(8);
    T jy = PS.h(2);
    jy = jy - PS.h(4);
    jy = jy + PS.h(5);
    jy = jy + PS.h(6);
    jy = jy - PS.h(7);
    jy = jy - PS.h(8);
    const T r = m.rho;
    const T mu = chi(m.fs, ps, c.mu), kth = chi(m.fs, ps, c.kth);
    const T sig = chi(m.fs, ps, c.sig), cp = chi(m.fs, ps, c.cp);
    const T mdot = c.one_m_rsl * (m.fs - fs_prev);                 // Eq. (ns1)
    // Single precision evaluates the collisions in an algebraically equal
    // form with the 1/c_s^2 factors folded (c_s^2 = 1/3), shared terms
    // hoisted and one reciprocal per divisor; double precision keeps the
    // printed operation order.
    constexpr bool FAST = sizeof(T) == 4;
    const T ir = FAST ? T(1) / r : T(0);
    const T usx = FAST ? (jx + T(0.5) * Fx) * ir : (jx + T(0.5) * Fx) / r;
    const T usy = FAST ? (jy + T(0.5) * Fy) * ir : (jy + T(0.5) * Fy) / r;
    const T fx = m.fs * (T(0) - usx), fy = m.fs * (T(0) - usy);    // u_s = 0
    const T ux = usx + T(0.5) * fx, uy = usy + T(0.5) * fy;        // Eq. (Computed_u)
    const T rfx = r * fx, rfy = r * fy;
    const T Sn = r * mdot + (ux * grhox + uy * grhoy);
    const T Ftx = Fx - gpx + cs2<T>() * grhox + cs2<T>() * gSx;
    const T Fty = Fy - gpy + cs2<T>() * grhoy + cs2<T>() * gSy;
    const T uF = ux * Ftx + uy * Fty;
    const T R0 = w9<T>(0) * (Sn - uF / cs2<T>());
    const T tau_h = FAST ? T(3) * mu * ir + T(0.5) : mu / r / cs2<T>() + T(0.5);
    T sh_ = T(0);
#pragma unroll
    for (int i = 1; i < 9; i++) sh_ += PS.h(i);
    const T p = cs2<T>() / (T(1) - w9<T>(0)) * (sh_ + T(0.5) * Sn + tau_h * R0 + r * s_i<T>(0, ux, uy));

    // ---- collisions + in-place streaming ---------------------------------
    const int xm = (x == 0) ? nx - 1 : x - 1, xp = (x == nx - 1) ? 0 : x + 1;
    const T uu_ = ux * ux + uy * uy;
    const T B15 = T(1.5) * uu_;                    // u.u / (2 c_s^2)

    // a7: flow
    {
        const T om = T(1) / tau_h;
        const T pre = FAST ? T(1) - T(0.5) * om : T(1) - T(1) / (T(2) * tau_h);
        auto put = [&](int i, T post) {
            bool wall;
            const uint32_t d = aa_dst<9, EDGE>(PH, i, P, pitch, x, y, xm, xp, ny, wall);
            Pol<S, T>::st(io.h + d, post, T(0), sh.h_scale);   // walls: half-way bounce-back
        };
        if constexpr (FAST) {
            // the rest direction, then every direction with its opposite:
            // the parts of h_eq and R_i even in c_i are shared by the pair,
            // the odd parts change sign
            const T omc = T(1) - om;
            const T A3 = T(3) * p;                      // p / c_s^2
            const T S3 = Sn - T(3) * uF;                // S - u.F~ / c_s^2
            const T Gx = Fx + rfx, Gy = Fy + rfy;
            const T base = A3 - r * B15;
            put(0, omc * PS.h(0) + om * (w9<T>(0) * base - A3) + pre * (w9<T>(0) * S3));
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int i = PAIR9[j], o = OPP9[i];
                const T w = w9<T>(i);
                const T cu = cdot<T>(CX[i], CY[i], ux, uy);
                const T cF = cdot<T>(CX[i], CY[i], Ftx, Fty);
                const T cG = cdot<T>(CX[i], CY[i], Gx, Gy);
                // h_eq = w (A3 + r (3 c.u + 4.5 (c.u)^2 - B15)), R_i = w (S3 + 3 c.G + 9 (c.u)(c.F~))
                const T ev = om * (w * (base + T(4.5) * r * cu * cu)) + pre * (w * (S3 + T(9) * cu * cF));
                const T od = om * (T(3) * w * r * cu) + pre * (T(3) * w * cG);
                put(i, omc * PS.h(i) + (ev + od));
                put(o, omc * PS.h(o) + (ev - od));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const T cu = cdot<T>(CX[i], CY[i], ux, uy);
                const T cF = cdot<T>(CX[i], CY[i], Ftx, Fty);
                const T Ri = w9<T>(i) * (Sn + cdot<T>(CX[i], CY[i], Fx + rfx, Fy + rfy) / cs2<T>() +
                                         (cu * cF - cs2<T>() * uF) / (cs2<T>() * cs2<T>()));
                const T heq = ((i == 0) ? p / cs2<T>() * (w9<T>(0) - T(1)) : p / cs2<T>() * w9<T>(i)) +
                              r * s_i<T>(i, ux, uy);
                put(i, PS.h(i) - (PS.h(i) - heq) / tau_h + pre * Ri);
            }
        }
    }
    // a5: phase field
    {
        const T pux = ps * ux, puy = ps * uy;
        const T dtx = pux - pux_prev;         // Euler d_t(psi u) (Sec. 3.4)
        const T dty = puy - puy_prev;
        pux_prev = pux;
        puy_prev = puy;
        // interface normal, regularised where grad psi vanishes (Sec. 2)
        const T gn = sqrt(gpsix * gpsix + gpsiy * gpsiy);
        const T ign = FAST ? T(1) / (gn + T(1e-4)) : T(0);
        const T nxv = FAST ? gpsix * ign : gpsix / (gn + T(1e-4));
        const T nyv = FAST ? gpsiy * ign : gpsiy / (gn + T(1e-4));
        const T lam = FAST ? c.four_over_W * ps * (T(1) - ps) : T(4) * ps * (T(1) - ps) / c.W;
        const T pre = FAST ? c.pre_f : T(1) - T(1) / (T(2) * c.tau_f);
        const T ax = dtx + cs2<T>() * lam * nxv;
        const T ay = dty + cs2<T>() * lam * nyv;
        const T om = FAST ? c.om_f : T(1) / c.tau_f;
        const T pmd = ps * mdot;
        uint32_t rb[4] = {0u, 0u, 0u, 0u};
        if constexpr (Pol<typename FStore<S>::type, T>::shifted) sr_block(rb, k, io.sr_step, 0u);
        auto put = [&](int i, T post) {
            bool wall;
            const uint32_t d = aa_dst<9, EDGE>(PH, i, P, pitch, x, y, xm, xp, ny, wall);
            T ref = T(0);
            if constexpr (Pol<typename FStore<S>::type, T>::shifted) {
                make_refs<S, T>(ro, sh, c, wall ? y : y + CY[i], ny);
                ref = wall ? ro.f[OPP9[i]] : ro.f[i];
            }
            Pol<typename FStore<S>::type, T>::st_sr(io.f + d, post, ref, sh.f_scale, bits13(rb, i));
        };
        if constexpr (FAST) {
            // f_eq = w psi (1 + 3 c.u), F_i = w (3 c.a + psi mdot): even parts
            // w (om psi + pre psi mdot) per weight, odd parts 3 w (om psi c.u + pre c.a)
            const T omc = T(1) - om;
            const T evw = om * ps + pre * pmd;
            put(0, omc * PS.f(0) + w9<T>(0) * evw);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int i = PAIR9[j], o = OPP9[i];
                const T w = w9<T>(i);
                const T ev = w * evw;
                const T od = T(3) * w * (om * ps * cdot<T>(CX[i], CY[i], ux, uy) + pre * cdot<T>(CX[i], CY[i], ax, ay));
                put(i, omc * PS.f(i) + (ev + od));
                put(o, omc * PS.f(o) + (ev - od));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const T cu = cdot<T>(CX[i], CY[i], ux, uy);
                const T feq = w9<T>(i) * ps * (T(1) + cu / cs2<T>());
                const T Fi = w9<T>(i) * cdot<T>(CX[i], CY[i], ax, ay) / cs2<T>() + w9<T>(i) * ps * mdot;
                put(i, PS.f(i) - (PS.f(i) - feq) / c.tau_f + pre * Fi);
            }
        }
    }
    // a8: enthalpy (Sec. 3.3)
    T Qn;
    {
        const T tau_g = FAST ? kth * ir * c.three_over_Cref + T(0.5) : kth / (r * c.Cref * cs2<T>()) + T(0.5);
        Qn = r * cp * m.T_ * mdot;
        const T uu = uu_;
        const T om = T(1) / tau_g;
        const T pre = FAST ? T(1) - T(0.5) * om : T(1) - T(1) / (T(2) * tau_g);
        const T CT = c.Cref * m.T_, cpT = cp * m.T_;
        uint32_t rb[4] = {0u, 0u, 0u, 0u};
        if constexpr (Pol<S, T>::shifted) sr_block(rb, k, io.sr_step, 2u);
        auto put = [&](int i, T post) {
            bool wall;
            const uint32_t d = aa_dst<9, EDGE>(PH, i, P, pitch, x, y, xm, xp, ny, wall);
            // cold wall: anti-bounce-back to C_p,ref T_w; top wall: adiabatic bounce-back
            const T val = (wall && y + CY[i] < 0) ? -post + T(2) * w9<T>(i) * c.Cref_Tw : post;
            T ref = T(0);
            if constexpr (Pol<S, T>::shifted) {
                make_refs<S, T>(ro, sh, c, wall ? y : y + CY[i], ny);
                ref = wall ? ro.g[OPP9[i]] : ro.g[i];
            }
            Pol<S, T>::st_sr(io.g + d, val, ref, sh.g_scale, bits13(rb, i));
        };
        if constexpr (FAST) {
            // g_eq = w (C T + C_p T (3 c.u + 4.5 (c.u)^2 - B15)): even part
            // shared by a direction and its opposite, odd part 3 w C_p T c.u
            const T omc = T(1) - om;
            const T base = CT - cpT * B15;
            put(0, omc * PS.g(0) + om * (m.H - CT + w9<T>(0) * base) + pre * (w9<T>(0) * Qn));
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int i = PAIR9[j], o = OPP9[i];
                const T w = w9<T>(i);
                const T cu = cdot<T>(CX[i], CY[i], ux, uy);
                const T ev = om * (w * (base + T(4.5) * cpT * cu * cu)) + pre * (w * Qn);
                const T od = om * (T(3) * w * cpT * cu);
                put(i, omc * PS.g(i) + (ev + od));
                put(o, omc * PS.g(o) + (ev - od));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const T cu = cdot<T>(CX[i], CY[i], ux, uy);
                T geq;
                if (i == 0)
                    geq = m.H - c.Cref * m.T_ + w9<T>(0) * cp * m.T_ * (c.Cref / cp - uu / (T(2) * cs2<T>()));
                else
                    geq = w9<T>(i) * cp * m.T_ *
                          (c.Cref / cp + cu / cs2<T>() + (cu * cu - cs2<T>() * uu) / (T(2) * cs2<T>() * cs2<T>()));
                put(i, PS.g(i) - (PS.g(i) - geq) / tau_g + pre * (w9<T>(i) * Qn));
            }
        }
    }
    // a6: potential (Sec. 3.4), one sweep inside the fused step (l has its
    // own layout phase, io.lph)
    {
        const T tau_l = FAST ? T(3) * sig + T(0.5) : sig / cs2<T>() + T(0.5);
        const T om = T(1) / tau_l;
        uint32_t rb[4] = {0u, 0u, 0u, 0u};
        if constexpr (Pol<S, T>::shifted) sr_block(rb, k, io.sr_step, 3u);
#pragma unroll
        for (int i = 0; i < 5; i++) {
            const T leq = (i == 0) ? (w5<T>(0) - T(1)) * m.phi : w5<T>(i) * m.phi;
            T post;
            if constexpr (FAST)
                post = PS.l(i) + om * (leq - PS.l(i));
            else
                post = PS.l(i) - (PS.l(i) - leq) / tau_l;
            bool wall;
            const uint32_t d = aa_dst<5, EDGE>(io.lph, i, P, pitch, x, y, xm, xp, ny, wall);
            T val = post;
            if (wall) {                           // electrodes: anti-bounce-back
                const T phiw = (y + CY5[i] < 0) ? c.phi_bot : c.phi_top;
                val = -post + T(2) * w5<T>(i) * phiw;
            }
            T ref = T(0);
            if constexpr (Pol<S, T>::shifted) {
                make_refs<S, T>(ro, sh, c, wall ? y : y + CY5[i], ny);
                ref = wall ? ro.l[OPP5[i]] : ro.l[i];
            }
            Pol<S, T>::st_sr(io.l + d, val, ref, sh.l_scale, bits13(rb, i));
        }
    }
    // previous-step fields for the next step
    io.aux_out[AUX_FS * P + k] = A(m.fs);
    io.aux_out[AUX_MDOT * P + k] = A(mdot);
    io.aux_out[AUX_Q * P + k] = A(Qn);
    io.aux_out[AUX_PUX * P + k] = A(pux_prev);
    io.aux_out[AUX_PUY * P + k] = A(puy_prev);
    io.aux_out[AUX_P * P + k] = A(p);
    io.aux_out[AUX_S * P + k] = A(Sn);
    if (io.write_sigma) io.sigma[k] = A(sig);
    if constexpr (!std::is_same<OB, NoObs>::value) ob->cell(io, c, sm, tx, ty, x, y, k, m, qv);
}


// One 32 x BY tile at (x0, y0) from layout phase PH (l: io.lph).
// ASYNC: the own cell's populations reach the stash by cp.async while the
// ring cell's loads are in flight (FP32 and FP64; half storage decodes its
// values in registers).  EARLY: the kernel was
// launched as a dependent of k_halo and has not waited for it yet; a full
// row in the natural layout is then copied from L2 (bypassing L1, whose
// lines may predate the step before) before the wait, so the copies overlap
// the end of k_halo, and everything else is read after it.
template <typename S, typename T, typename A, int BY, int PH, bool ASYNC = false, typename OB = NoObs,
          bool EARLY = false>
__device__ __forceinline__ void step_tile(const StepIO<S, T, A> &io, const Consts<T> &c,
                                          const Shift &sh, TileSmem<T, BY> &sm, T (*stash)[BY][32], int x0,
                                          int y0, OB *ob = nullptr) {
    constexpr bool OBS = !std::is_same<OB, NoObs>::value;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const int nx = io.nx, ny = io.ny;
    const uint32_t P = (uint32_t)io.plane;   // 32-bit offsets (checked at creation)
    const uint32_t pitch = (uint32_t)io.pitch;

    // columns of this tile: 32, or fewer on a ragged last tile, where the
    // lane right after the last column holds the wrap-around neighbour x = 0
    const int ncols = nx - x0 < 32 ? nx - x0 : 32;
    const int y = y0 + ty;
    const bool own = tx < ncols && y < ny;
    const bool wrap = tx == ncols && y < ny;     // only when ncols < 32
    const int x = own ? x0 + tx : 0;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const uint32_t k = (uint32_t)y * pitch + (uint32_t)x;
    Macro<T> m;
    T fs_prev = T(0), mdot_prev = T(0), Q_prev = T(0), pux_prev = T(0), puy_prev = T(0);
    constexpr int NRING = 2 * 34 + 2 * BY;
    static_assert(NRING <= 32 * BY, "one ring cell per thread at most");
    // the ring slot of this thread, if any: rows beyond a wall are ghosts,
    // and on a ragged tile only columns up to the wrap-around one are used
    int rex = 0, rey = 0, rhx = 0, rhy = 0;
    bool ring = false;
    if (tid < NRING) {
        ring_slot<BY>(tid, rex, rey);
        rhy = y0 - 1 + rey;
        // x0 - 1 + ex lies in [-1, nx]: -1 and nx wrap around
        const int hx = x0 - 1 + rex;
        rhx = hx < 0 ? hx + nx : (hx >= nx ? hx - nx : hx);
        ring = rhy >= 0 && rhy < ny && rex <= ncols + 1;
    }
    if constexpr (ASYNC && std::is_same<S, T>::value && std::is_same<typename FStore<S>::type, S>::value) {
        // ---- phase 1, FP32/FP64: the own cells' populations go straight
        // from global to the stash (cp.async, no registers), the ring cell's
        // loads are issued meanwhile, so both wait for memory once
        T pv = T(0), Sv = T(0);
        const bool early = EARLY && PH == 0 && ncols == 32 && io.lph == 0;
        if (EARLY && !early) grid_dep_wait();
        if (own) {
            if (early) {
                stash_row_async<T, BY, true>(stash, ty, tx, io.f, io.l, P, (uint32_t)y * pitch + (uint32_t)x0, true);
            } else if (PH == 0 && ncols == 32) {
                // natural layout, full row: each warp copies its row in
                // 16-byte chunks (l_1..4 gathered if l is swapped)
                stash_row_async<T, BY>(stash, ty, tx, io.f, io.l, P, (uint32_t)y * pitch + (uint32_t)x0,
                                       io.lph == 0);
                if (io.lph != 0) {
#pragma unroll
                    for (int i = 1; i < 5; i++)
                        cp_async_elem(&stash[27 + i][ty][tx], io.l + aa_src<5>(1, i, P, pitch, x, y, xm, xp, ny));
                }
            } else {          // swapped layout or ragged tile: one element each
#pragma unroll
                for (int i = 0; i < 9; i++) {
                    const uint32_t o9 = aa_src<9>(PH, i, P, pitch, x, y, xm, xp, ny);
                    cp_async_elem(&stash[i][ty][tx], io.f + o9);
                    cp_async_elem(&stash[9 + i][ty][tx], io.h + o9);
                    cp_async_elem(&stash[18 + i][ty][tx], io.g + o9);
                }
#pragma unroll
                for (int i = 0; i < 5; i++)
                    cp_async_elem(&stash[27 + i][ty][tx], io.l + aa_src<5>(io.lph, i, P, pitch, x, y, xm, xp, ny));
            }
            if (early) {
                pux_prev = T(__ldcg(io.aux_in + (AUX_PUX * P + k)));
                puy_prev = T(__ldcg(io.aux_in + (AUX_PUY * P + k)));
                fs_prev = T(__ldcg(io.aux_in + (AUX_FS * P + k)));
                mdot_prev = T(__ldcg(io.aux_in + (AUX_MDOT * P + k)));
                Q_prev = T(__ldcg(io.aux_in + (AUX_Q * P + k)));
                pv = T(__ldcg(io.aux_in + (AUX_P * P + k)));
                Sv = T(__ldcg(io.aux_in + (AUX_S * P + k)));
            } else {
                pux_prev = T(io.aux_in[AUX_PUX * P + k]);
                puy_prev = T(io.aux_in[AUX_PUY * P + k]);
                fs_prev = T(io.aux_in[AUX_FS * P + k]);
                mdot_prev = T(io.aux_in[AUX_MDOT * P + k]);
                Q_prev = T(io.aux_in[AUX_Q * P + k]);
                pv = T(io.aux_in[AUX_P * P + k]);
                Sv = T(io.aux_in[AUX_S * P + k]);
            }
        }
        if (EARLY && early) grid_dep_wait();      // k_halo's records
        RingLoad<T> rl;
        if (ring) ring_load(io, rhx, rhy, rl);
        if (own) {
            cp_async_wait_all();
            if (ncols == 32) __syncwarp();   // a full row's planes were copied by the whole warp
            T f[9], g[9];
#pragma unroll
            for (int i = 0; i < 9; i++) {
                f[i] = stash[i][ty][tx];
                g[i] = stash[18 + i][ty][tx];
            }
            T l1234 = stash[28][ty][tx];
            l1234 = l1234 + stash[29][ty][tx];
            l1234 = l1234 + stash[30][ty][tx];
            l1234 = l1234 + stash[31][ty][tx];
            local_macros(f, g, l1234, fs_prev, mdot_prev, Q_prev, c, m);
            sm.q[ty + 1][tx + 1] = {m.psi, m.rho, m.eps, m.phi};
            sm.ps[ty + 1][tx + 1] = {pv, Sv};
            if constexpr (OBS) ob->macro(ty + 1, tx + 1, m);
        }
        if (ring) ring_to_smem<T, BY, OB>(c, rl, sm, rex, rey, ob);
    } else {
        // ---- phase 1: own cell (kept in registers) -------------------------
        Refs<T> rf;
        T f[9], g[9], l[5], h[9];
        const float fsc = 1.0f / sh.f_scale, gsc = 1.0f / sh.g_scale, lsc = 1.0f / sh.l_scale;
        const float hsc = 1.0f / sh.h_scale;
        if (own) {
            make_refs<S, T>(rf, sh, c, y, ny);
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const uint32_t o9 = aa_src<9>(PH, i, P, pitch, x, y, xm, xp, ny);
                f[i] = Pol<typename FStore<S>::type, T>::ld(io.f + o9, rf.f[i], fsc);
                g[i] = Pol<S, T>::ld(io.g + o9, rf.g[i], gsc);
                h[i] = Pol<S, T>::ld(io.h + o9, T(0), hsc);
            }
#pragma unroll
            for (int i = 0; i < 5; i++)
                l[i] = Pol<S, T>::ld(io.l + aa_src<5>(io.lph, i, P, pitch, x, y, xm, xp, ny), rf.l[i], lsc);
            pux_prev = T(io.aux_in[AUX_PUX * P + k]);
            puy_prev = T(io.aux_in[AUX_PUY * P + k]);
            fs_prev = T(io.aux_in[AUX_FS * P + k]);
            mdot_prev = T(io.aux_in[AUX_MDOT * P + k]);
            Q_prev = T(io.aux_in[AUX_Q * P + k]);
            T l1234 = T(0);
#pragma unroll
            for (int i = 1; i < 5; i++) l1234 += l[i];
            local_macros(f, g, l1234, fs_prev, mdot_prev, Q_prev, c, m);
            // keep the populations for phase 2 in shared memory, not registers
#pragma unroll
            for (int i = 0; i < 9; i++) {
                stash[i][ty][tx] = f[i];
                stash[9 + i][ty][tx] = h[i];
                stash[18 + i][ty][tx] = g[i];
            }
#pragma unroll
            for (int i = 0; i < 5; i++) stash[27 + i][ty][tx] = l[i];
            sm.q[ty + 1][tx + 1] = {m.psi, m.rho, m.eps, m.phi};
            sm.ps[ty + 1][tx + 1] = {T(io.aux_in[AUX_P * P + k]), T(io.aux_in[AUX_S * P + k])};
            if constexpr (OBS) ob->macro(ty + 1, tx + 1, m);
        }
        // ---- phase 1: halo ring, from the halo records
        if (ring) {
            RingLoad<T> rl;
            ring_load(io, rhx, rhy, rl);
            ring_to_smem<T, BY, OB>(c, rl, sm, rex, rey, ob);
        }
    }
    // the wrap-around neighbour of a ragged tile's last column
    if (wrap) {
        RingLoad<T> rl;
        ring_load(io, 0, y, rl);
        ring_to_smem<T, BY, OB>(c, rl, sm, tx + 1, ty + 1, ob);
    }
    __syncthreads();
    fill_ghosts<T, BY>(sm, c, y0, ny, tid);
    __syncthreads();
    if (!own) return;
    const StashPops<T, BY> PS{stash, ty, tx};
    if (y0 == 0 || y0 + BY >= ny)
        step_cell<S, T, A, BY, true, PH>(io, c, sh, sm, PS, tx, ty, x, y, m, fs_prev, pux_prev, puy_prev, ob);
    else
        step_cell<S, T, A, BY, false, PH>(io, c, sh, sm, PS, tx, ty, x, y, m, fs_prev, pux_prev, puy_prev, ob);
}

// Blocks per SM the single-precision step asks the register allocator for:
// with 4-row tiles, 7 blocks (28 warps) hold a 512 x 256 lattice in one wave.
// (8 blocks at 64 registers were 0.3 us faster at 1024 x 512 but slowed the
// one-wave lattices: latency per block counts there.)
template <typename S, typename T, int BY>
constexpr int step_min_blocks() {
    return sizeof(T) == 8 ? 1 : (BY == 4 ? 7 : (BY == 8 ? 4 : 1));
}

// Blocks per SM of the batched step: fewer than the single-instance step's,
// so its extra live state (the member's constants and work-list position)
// fits in registers without spills (measured on the 64-instance mix: 1.49x
// over plain against 1.23x with 7 blocks and spills).
template <typename T, int BY>
constexpr int batch_min_blocks() {
    return sizeof(T) == 8 ? 1 : (BY == 4 ? 5 : (BY == 8 ? 3 : 1));
}

template <typename T, int BY>
constexpr size_t stash_bytes() { return size_t(NPOP) * BY * 32 * sizeof(T); }

// Opt a kernel into its dynamic shared memory once per device: `done` holds
// one bit per device ordinal (the attribute is per device), so handles on
// several GPUs and threads holding different handles are served.
template <typename K>
inline cudaError_t allow_dynamic_smem(K kernel, size_t bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// io: step_io() of this launch's parities, resolved on the host (PH = cur).
template <typename S, typename T, typename A, int BY, int PH>
__global__ void __launch_bounds__(32 * BY, step_min_blocks<S, T, BY>())
    k_step(StepIO<S, T, A> io, Consts<T> c, Shift sh) {
    __shared__ TileSmem<T, BY> sm;
    extern __shared__ __align__(16) unsigned char dsm_stash[];     // NPOP x BY x 32 values
    T(*stash)[BY][32] = reinterpret_cast<T(*)[BY][32]>(dsm_stash);
    // FP32 and FP64 wait for k_halo inside step_tile (after copying what
    // does not depend on it); half storage reads its rounding counter first
    constexpr bool EARLY = std::is_same<S, T>::value && std::is_same<typename FStore<S>::type, S>::value;
    if constexpr (!EARLY) grid_dep_wait();
    grid_dep_release();                // the next step's k_halo waits for this grid's end
    load_counters(io, PH);
    advance_counters(io, PH, blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0);
    step_tile<S, T, A, BY, PH, true, NoObs, EARLY>(io, c, sh, sm, stash, blockIdx.x * 32, blockIdx.y * BY);
}

// The tile-edge cells of the 32 x BY tile at (x0, y0), one per thread of a
// HALO_THREADS block: its bottom and top rows, then the inner cells of its
// first and last columns.
constexpr int HALO_THREADS = 96;
// Blocks per SM the halo kernels ask the register allocator for: each
// thread only loads and sums, so many blocks keep more loads in flight.
template <typename T>
constexpr int halo_min_blocks() { return sizeof(T) == 8 ? 8 : 16; }
template <typename S, typename T, typename A, int BY, int PH>
__device__ __forceinline__ void halo_tile(const StepIO<S, T, A> &io, const Consts<T> &c, const Shift &sh, int x0,
                                          int y0, int j) {
    static_assert(2 * 32 + 2 * (BY - 2) <= HALO_THREADS, "one edge cell per thread");
    const int ncols = io.nx - x0 < 32 ? io.nx - x0 : 32;
    int tx, ty;
    if (j < ncols) {
        tx = j;
        ty = 0;
    } else if (j < 2 * ncols) {
        tx = j - ncols;
        ty = BY - 1;
    } else {
        const int r = j - 2 * ncols;
        if (r < BY - 2) {
            tx = 0;
            ty = 1 + r;
        } else if (r < 2 * (BY - 2) && ncols > 1) {
            tx = ncols - 1;
            ty = 1 + r - (BY - 2);
        } else {
            return;
        }
    }
    const int y = y0 + ty;
    if (y >= io.ny) return;
    halo_cell<S, T, A, PH>(io, c, sh, x0 + tx, y);
}

// First launch of a step: the halo records of every tile-edge cell, from
// the populations the step before left (layout phase PH, l: io.lph).
template <typename S, typename T, typename A, int BY, int PH>
__global__ void __launch_bounds__(HALO_THREADS, halo_min_blocks<T>()) k_halo(StepIO<S, T, A> io, Consts<T> c,
                                                                             Shift sh) {
    grid_dep_wait();                   // the populations of the step before
    grid_dep_release();
    halo_tile<S, T, A, BY, PH>(io, c, sh, blockIdx.x * 32, blockIdx.y * BY, threadIdx.x);
}

// Batched form: blocks walk a flat list of tiles of many instances.  The
// parities of every member flip together, so the list keeps each member's
// parity at the start and the launch passes the flips since then.
template <bool SWEEP>
__device__ __forceinline__ int find_item(const BatchItem *__restrict__ items, int n_items, int t) {
    int lo = 0, hi = n_items - 1;      // last item whose first tile is <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b = SWEEP ? items[mid].sweep_begin : items[mid].tile_begin;
        if (b <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename S, typename T, typename A, int BY>
__global__ void __launch_bounds__(32 * BY, batch_min_blocks<T, BY>()) k_batch_step(const BatchItem *__restrict__ items,
                                                        const Consts<T> *__restrict__ consts,
                                                        const int *__restrict__ tile_item, int total_tiles,
                                                        int flip_cur, int flip_l) {
    __shared__ TileSmem<T, BY> sm;
    extern __shared__ __align__(16) unsigned char dsm_stash[];     // NPOP x BY x 32 values
    T(*stash)[BY][32] = reinterpret_cast<T(*)[BY][32]>(dsm_stash);
    __shared__ Consts<T> s_c;          // the member's constants, staged once per tile
    constexpr int NC = int(sizeof(Consts<T>) / sizeof(T));
    static_assert(sizeof(Consts<T>) == NC * sizeof(T), "Consts holds only T");
    const int tid = threadIdx.y * 32 + threadIdx.x;
    grid_dep_wait();
    grid_dep_release();
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const int item = tile_item[t];
        if (tid < NC) reinterpret_cast<T *>(&s_c)[tid] = reinterpret_cast<const T *>(consts + item)[tid];
        __syncthreads();
        const BatchItem &it = items[item];
        const int local = t - it.tile_begin;
        const int bx = local % it.tiles_x, by = local / it.tiles_x;
        const int cur = it.cur ^ flip_cur;
        StepIO<S, T, A> io = step_io<S, T, A>(it.s, cur, it.lcur ^ flip_l, it.write_sigma);
        load_counters(io, cur);
        advance_counters(io, cur, local == 0 && tid == 0);
        if (cur)
            step_tile<S, T, A, BY, 1, true>(io, s_c, it.sh, sm, stash, bx * 32, by * BY);
        else
            step_tile<S, T, A, BY, 0, true>(io, s_c, it.sh, sm, stash, bx * 32, by * BY);
        __syncthreads();
    }
}

// Batched form of k_halo over the same work list.
template <typename S, typename T, typename A, int BY>
__global__ void __launch_bounds__(HALO_THREADS, halo_min_blocks<T>()) k_batch_halo(const BatchItem *__restrict__ items,
                                                             const Consts<T> *__restrict__ consts,
                                                             const int *__restrict__ tile_item, int total_tiles,
                                                             int flip_cur, int flip_l) {
    grid_dep_wait();
    grid_dep_release();
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const int item = tile_item[t];
        const BatchItem &it = items[item];
        const int local = t - it.tile_begin;
        const int bx = local % it.tiles_x, by = local / it.tiles_x;
        const int cur = it.cur ^ flip_cur;
        const StepIO<S, T, A> io = step_io<S, T, A>(it.s, cur, it.lcur ^ flip_l, it.write_sigma);
        if (cur)
            halo_tile<S, T, A, BY, 1>(io, consts[item], it.sh, bx * 32, by * BY, threadIdx.x);
        else
            halo_tile<S, T, A, BY, 0>(io, consts[item], it.sh, bx * 32, by * BY, threadIdx.x);
    }
}

// ---------------------------------------------------------------------------
// Extra potential sweeps (k_e > 1 and the pre-solve): D2Q5 collide with sigma
// frozen at time n, streamed in place from layout phase lph, anti-bounce-back
// at the electrodes.  Purely local: no halo, so no publication is needed.
// ---------------------------------------------------------------------------
template <typename S, typename T, typename A>
__device__ __forceinline__ void sweep_cell(S *l, const A *sigma, int nx, int ny, int pitch, uint32_t P,
                                           const Consts<T> &c, const Shift &sh, int x, int y, int lph,
                                           uint32_t sr_step, uint32_t sr_sys) {
    const uint32_t k = (uint32_t)y * (uint32_t)pitch + (uint32_t)x;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    // half storage rounds stochastically here too: rounding to nearest would
    // stall the relaxation once a sweep changes phi by less than half a
    // spacing (sr_sys keeps every sweep's bits apart from the step's)
    uint32_t rb[4] = {0u, 0u, 0u, 0u};
    if constexpr (Pol<S, T>::shifted) sr_block(rb, k, sr_step, sr_sys);
    Refs<T> rf, ro;
    make_refs<S, T>(rf, sh, c, y, ny);
    const float lsc = 1.0f / sh.l_scale;
    T lv[5];
#pragma unroll
    for (int i = 0; i < 5; i++)
        lv[i] = Pol<S, T>::ld(l + aa_src<5>(lph, i, P, (uint32_t)pitch, x, y, xm, xp, ny), rf.l[i], lsc);
    T sl = T(0);
#pragma unroll
    for (int i = 1; i < 5; i++) sl += lv[i];
    const T phi = sl / (T(1) - w5<T>(0));
    const T tau_l = T(sigma[k]) / cs2<T>() + T(0.5);
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const T leq = (i == 0) ? (w5<T>(0) - T(1)) * phi : w5<T>(i) * phi;
        const T post = lv[i] - (lv[i] - leq) / tau_l;
        bool wall;
        const uint32_t d = aa_dst<5, true>(lph, i, P, (uint32_t)pitch, x, y, xm, xp, ny, wall);
        T val = post;
        if (wall) {
            const T phiw = (y + CY5[i] < 0) ? c.phi_bot : c.phi_top;
            val = -post + T(2) * w5<T>(i) * phiw;
        }
        T ref = T(0);
        if constexpr (Pol<S, T>::shifted) {
            make_refs<S, T>(ro, sh, c, wall ? y : y + CY5[i], ny);
            ref = wall ? ro.l[OPP5[i]] : ro.l[i];
        }
        Pol<S, T>::st_sr(l + d, val, ref, sh.l_scale, bits13(rb, i));
    }
}

// lcur: the layout phase of l; cur: the population parity, whose rounding
// counter (half storage) the sweep reads; sr_sys: this sweep's rounding stream.
template <typename S, typename T, typename A>
__global__ void k_sweep(DevState s, int lcur, int cur, uint32_t sr_sys, Consts<T> c, Shift sh) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= s.nx || y >= s.ny) return;
    S *l = Planes<S>::at(s.pop, s.plane).l;
    const uint32_t sr_step = (Pol<S, T>::shifted && s.rng) ? s.rng[cur] : 0u;
    sweep_cell<S, T, A>(l, reinterpret_cast<const A *>(s.sigma), s.nx, s.ny, s.pitch, (uint32_t)s.plane, c, sh, x, y,
                        lcur, sr_step, sr_sys);
}

// Batched potential sweep over the same work list (32 x 8 cells per tile).
template <typename S, typename T, typename A>
__global__ void __launch_bounds__(256) k_batch_sweep(const BatchItem *__restrict__ items,
                                                     const Consts<T> *__restrict__ consts, int n_items,
                                                     int total_tiles, int flip_l, int flip_cur,
                                                     uint32_t sr_sys) {
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const int ii = find_item<true>(items, n_items, t);
        const BatchItem &it = items[ii];
        const int local = t - it.sweep_begin;
        const int x = (local % it.sweep_tiles_x) * 32 + threadIdx.x;
        const int y = (local / it.sweep_tiles_x) * 8 + threadIdx.y;
        if (x < it.s.nx && y < it.s.ny) {
            S *l = Planes<S>::at(it.s.pop, it.s.plane).l;
            const uint32_t sr_step = (Pol<S, T>::shifted && it.s.rng) ? it.s.rng[it.cur ^ flip_cur] : 0u;
            sweep_cell<S, T, A>(l, reinterpret_cast<const A *>(it.s.sigma), it.s.nx, it.s.ny, it.s.pitch,
                                (uint32_t)it.s.plane, consts[ii], it.sh, x, y, it.lcur ^ flip_l, sr_step, sr_sys);
        }
    }
}

// ---------------------------------------------------------------------------
// Initial state (Sec. 2): equilibria of a resting droplet at T_init with all
// latent heat held, linear potential between the electrodes; natural layout
// (phase 0).
// ---------------------------------------------------------------------------
template <typename S, typename T, typename A>
__global__ void k_init(DevState s, const double *psi_dev, double R, double xc, double yc, double W,
                       Consts<T> c, Shift sh) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= s.nx || y >= s.ny) return;
    const long long P = s.plane, k = (long long)y * s.pitch + x;
    double psd;
    if (psi_dev) {
        psd = psi_dev[(long long)y * s.nx + x];
    } else {
        const double dx = x - xc, dy = y - yc;
        const double rr = sqrt(dx * dx + dy * dy);
        psd = 0.5 + 0.5 * tanh(2.0 * (R - rr) / W);
    }
    const T ps = T(psd);
    const T cpm = chi(T(0), ps, c.cp);
    const T T0 = c.T_init;
    const T H0 = cpm * T0 + ps * c.L;
    const T phi0 = c.phi_bot + (c.phi_top - c.phi_bot) * (T(y) + T(0.5)) / T(s.ny);
    const T rho0 = chi(T(0), ps, c.rho);
    Refs<T> rf;
    make_refs<S, T>(rf, sh, c, y, s.ny);
    const Planes<S> pl = Planes<S>::at(s.pop, P);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const T feq = w9<T>(i) * ps * (T(1) + T(0) / cs2<T>());
        const T pre = (i == 0) ? T(0) / cs2<T>() * (w9<T>(0) - T(1)) : T(0) / cs2<T>() * w9<T>(i);
        const T heq = pre + rho0 * s_i<T>(i, T(0), T(0));
        T geq;
        if (i == 0)
            geq = H0 - c.Cref * T0 + w9<T>(0) * cpm * T0 * (c.Cref / cpm - T(0) / (T(2) * cs2<T>()));
        else
            geq = w9<T>(i) * cpm * T0 * (c.Cref / cpm + T(0) / cs2<T>() + (T(0) - T(0)) / (T(2) * cs2<T>() * cs2<T>()));
        Pol<typename FStore<S>::type, T>::st(pl.f + i * P + k, feq, rf.f[i], sh.f_scale);
        Pol<S, T>::st(pl.h + i * P + k, heq, T(0), sh.h_scale);
        Pol<S, T>::st(pl.g + i * P + k, geq, rf.g[i], sh.g_scale);
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const T leq = (i == 0) ? (w5<T>(0) - T(1)) * phi0 : w5<T>(i) * phi0;
        Pol<S, T>::st(pl.l + i * P + k, leq, rf.l[i], sh.l_scale);
    }
    A *aux = reinterpret_cast<A *>(s.aux[0]);
#pragma unroll
    for (int a = 0; a < NAUX; a++) aux[a * P + k] = A(0);
    reinterpret_cast<A *>(s.sigma)[k] = A(chi(T(0), ps, c.sig));
}

}  // namespace lbm
