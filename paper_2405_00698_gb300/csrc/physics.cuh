// Per-spring and per-mass arithmetic of one time step (Section II-C; Table II constants), shared
// by the lattice stepping kernel, the checkpoint replay of the adjoint and the adjoint itself.
// Every operation is an explicitly rounded intrinsic, so the compiler cannot contract or reorder
// it differently in different kernels: a replay from a checkpoint reproduces the forward run bit
// for bit, and the contact modes the adjoint holds fixed are the ones the forward run took.
#pragma once

#include "common.cuh"

namespace vx {

// (-1, -1): F - g for a pair as one fused multiply-add F + g * (-1), exact product, one rounding
// as the subtraction (the paired add takes no negated operand, so -g would cost two more
// instructions; 5 % fewer in the lattice step's backward gather).
constexpr float2 kMinusOne2 = {-1.f, -1.f};

// Force on the first endpoint a of a spring (the second endpoint b receives its negative).
//   du = u_b - u_a (displacements from the rest lattice), d = d0 + du with d0 the lattice
//   offset; from the cancellation-free numerator n = 2 d0.du + du.du, l^2 = L0^2 + n and the
//   extension e0 = l - L0 = n / (l + L0);
//   actuated rest length L = L0 + act with act = (alpha L0) sin(w t) + (beta L0) cos(w t);
//   f = k (l - L) d / l.
// Outputs the force g (on a), and for the adjoint the unit-free pieces ext = l - L and inv = 1/l.
struct SpringEval {
    float dx, dy, dz;   // spring vector a -> b
    float inv;          // 1 / l
    float ext;          // l - L
    float gx, gy, gz;   // force on a
};

// Spring along lattice direction D (compile-time): the zero components of the lattice offset d0
// drop out of the arithmetic statically.
template <int D>
__device__ __forceinline__ SpringEval spring_eval_dir(float dux, float duy, float duz, float edge,
                                                      float L0, float L0sq, float k, float pa, float pb,
                                                      float sn, float cs)
{
    constexpr int ox = lattice_dir(D, 0), oy = lattice_dir(D, 1), oz = lattice_dir(D, 2);
    SpringEval e;
    e.dx = ox ? __fadd_rn(ox > 0 ? edge : -edge, dux) : dux;
    e.dy = oy ? __fadd_rn(oy > 0 ? edge : -edge, duy) : duy;
    e.dz = oz ? __fadd_rn(oz > 0 ? edge : -edge, duz) : duz;
    // d0 . du over the non-zero components of d0 (each +-edge)
    float d0du = 0.0f;
    if (ox) d0du = __fmaf_rn(ox > 0 ? edge : -edge, dux, d0du);
    if (oy) d0du = __fmaf_rn(oy > 0 ? edge : -edge, duy, d0du);
    if (oz) d0du = __fmaf_rn(oz > 0 ? edge : -edge, duz, d0du);
    const float dudu = __fmaf_rn(duz, duz, __fmaf_rn(duy, duy, __fmul_rn(dux, dux)));
    const float num = __fmaf_rn(2.0f, d0du, dudu);
    const float l2 = __fadd_rn(L0sq, num);      // |d0 + du|^2 = L0^2 + 2 d0.du + du.du
    e.inv = rsqrtf(l2);
    const float l = __fmul_rn(l2, e.inv);
    const float act = __fmaf_rn(pa, sn, __fmul_rn(pb, cs));
    e.ext = __fsub_rn(__fdividef(num, __fadd_rn(l, L0)), act);
    const float f = l2 > 1e-30f ? __fmul_rn(__fmul_rn(k, e.ext), e.inv) : 0.0f;
    const float2 gxy = __fmul2_rn(make_float2(f, f), make_float2(e.dx, e.dy));
    e.gx = gxy.x;
    e.gy = gxy.y;
    e.gz = __fmul_rn(f, e.dz);
    return e;
}

// The same from the two endpoints' displacements (b: far end, a: this end): du's x and y lanes
// as one paired fused multiply-add b + a * (-1) (exact product, the subtraction's rounding).
// Used by the resident kernels (2.2 % fewer instructions in the lattice step); the streamed
// kernels, at 64 registers, measured slower with it and keep three subtractions.
template <int D>
__device__ __forceinline__ SpringEval spring_eval_ends(const float4& b, const float4& a, float edge, float L0,
                                                       float L0sq, float k, float pa, float pb, float sn, float cs)
{
    const float2 dxy = __ffma2_rn(make_float2(a.x, a.y), kMinusOne2, make_float2(b.x, b.y));
    return spring_eval_dir<D>(dxy.x, dxy.y, __fsub_rn(b.z, a.z), edge, L0, L0sq, k, pa, pb, sn, cs);
}

// The same spring evaluation for a lattice offset (ox, oy, oz) known only at run time.
__device__ __forceinline__ SpringEval spring_eval_rt(float dux, float duy, float duz, int ox, int oy, int oz,
                                                     float edge, float L0, float L0sq, float k, float pa,
                                                     float pb, float sn, float cs)
{
    SpringEval e;
    e.dx = ox ? __fadd_rn(ox > 0 ? edge : -edge, dux) : dux;
    e.dy = oy ? __fadd_rn(oy > 0 ? edge : -edge, duy) : duy;
    e.dz = oz ? __fadd_rn(oz > 0 ? edge : -edge, duz) : duz;
    float d0du = 0.0f;
    if (ox) d0du = __fmaf_rn(ox > 0 ? edge : -edge, dux, d0du);
    if (oy) d0du = __fmaf_rn(oy > 0 ? edge : -edge, duy, d0du);
    if (oz) d0du = __fmaf_rn(oz > 0 ? edge : -edge, duz, d0du);
    const float dudu = __fmaf_rn(duz, duz, __fmaf_rn(duy, duy, __fmul_rn(dux, dux)));
    const float num = __fmaf_rn(2.0f, d0du, dudu);
    const float l2 = __fadd_rn(L0sq, num);      // |d0 + du|^2 = L0^2 + 2 d0.du + du.du
    e.inv = rsqrtf(l2);
    const float l = __fmul_rn(l2, e.inv);
    const float act = __fmaf_rn(pa, sn, __fmul_rn(pb, cs));
    e.ext = __fsub_rn(__fdividef(num, __fadd_rn(l, L0)), act);
    const float f = l2 > 1e-30f ? __fmul_rn(__fmul_rn(k, e.ext), e.inv) : 0.0f;
    e.gx = __fmul_rn(f, e.dx);
    e.gy = __fmul_rn(f, e.dy);
    e.gz = __fmul_rn(f, e.dz);
    return e;
}

// Rest length of lattice direction D (compile-time class: edge, face or body diagonal).
template <int D>
__device__ __forceinline__ float lattice_rest(const StepConst& c)
{
    constexpr int cls = (lattice_dir(D, 0) != 0) + (lattice_dir(D, 1) != 0) + (lattice_dir(D, 2) != 0);
    return cls == 1 ? c.edge : (cls == 2 ? c.edge_sqrt2 : c.edge_sqrt3);
}

// Its square (edge^2 times 1, 2 or 3, each rounded once from the exact value).
template <int D>
__device__ __forceinline__ float lattice_rest_sq(const StepConst& c)
{
    constexpr int cls = (lattice_dir(D, 0) != 0) + (lattice_dir(D, 1) != 0) + (lattice_dir(D, 2) != 0);
    return cls == 1 ? c.edge_sq : (cls == 2 ? c.edge_sq2 : c.edge_sq3);
}

// The same for an offset known at run time.
__device__ __forceinline__ float lattice_rest_sq_rt(int ox, int oy, int oz, const StepConst& c)
{
    const int cls = (ox != 0) + (oy != 0) + (oz != 0);
    return cls == 1 ? c.edge_sq : (cls == 2 ? c.edge_sq2 : c.edge_sq3);
}

// Corner-index offset of lattice direction D on a grid with X corners per row and XY per layer.
template <int D>
__device__ __forceinline__ int lattice_offset(int X, int XY)
{
    return lattice_dir(D, 0) + X * lattice_dir(D, 1) + XY * lattice_dir(D, 2);
}

// Compile-time loop over the 13 directions: f(std::integral_constant-like tag).
template <int D>
struct DirTag {
    static constexpr int value = D;
};
template <int D = 0, class F>
__device__ __forceinline__ void for_each_dir(F&& f)
{
    if constexpr (D < 13) {
        f(DirTag<D>{});
        for_each_dir<D + 1>(f);
    }
}

// Directions D0 .. D0 + N - 1.
template <int D0, int N, class F>
__device__ __forceinline__ void for_each_dir_in(F&& f)
{
    if constexpr (N > 0) {
        f(DirTag<D0>{});
        for_each_dir_in<D0 + 1, N - 1>(f);
    }
}

// First directions of consecutive batches of B directions: 0, B, 2B, ... below 13.
template <int B, int D0 = 0, class F>
__device__ __forceinline__ void for_each_batch(F&& f)
{
    if constexpr (D0 < 13) {
        f(DirTag<D0>{});
        for_each_batch<B, D0 + B>(f);
    }
}

// Spring dashpot of the paper's preset (Table II spring damping ratio): adds
// c_s ((v_b - v_a) . u) u to the force on a, c_s = spring_c sqrt(k) (spring_c = 2 zeta sqrt(m / 2)).
__device__ __forceinline__ void spring_dashpot(SpringEval& e, float dvx, float dvy, float dvz, float k,
                                               const StepConst& c)
{
    const float cs = __fmul_rn(c.spring_c, __fsqrt_rn(k));
    const float rv = __fmul_rn(__fmaf_rn(e.dz, dvz, __fmaf_rn(e.dy, dvy, __fmul_rn(e.dx, dvx))), e.inv);
    const float fd = __fmul_rn(__fmul_rn(cs, rv), e.inv);      // per unit of d
    e.gx = __fmaf_rn(fd, e.dx, e.gx);
    e.gy = __fmaf_rn(fd, e.dy, e.gy);
    e.gz = __fmaf_rn(fd, e.dz, e.gz);
}

// Semi-implicit Euler with velocity damping, v <- c (v + dt F / m), u <- u + dt v, with the
// constants carried past float32 (see StepConst): w = v + (dt/m)_hi F + (dt/m)_lo F,
// v = w - (1 - c) w, u = u + dt_hi v + dt_lo v.
__device__ __forceinline__ void integrate(float4& u, float4& v, float Fx, float Fy, float Fz, const StepConst& c)
{
    const float wx = __fmaf_rn(c.dt_over_m, Fx, __fmaf_rn(c.dtm_lo, Fx, v.x));
    const float wy = __fmaf_rn(c.dt_over_m, Fy, __fmaf_rn(c.dtm_lo, Fy, v.y));
    const float wz = __fmaf_rn(c.dt_over_m, Fz, __fmaf_rn(c.dtm_lo, Fz, v.z));
    v.x = __fmaf_rn(-c.damping_c, wx, wx);
    v.y = __fmaf_rn(-c.damping_c, wy, wy);
    v.z = __fmaf_rn(-c.damping_c, wz, wz);
    u.x = __fmaf_rn(c.dt, v.x, __fmaf_rn(c.dt_lo, v.x, u.x));
    u.y = __fmaf_rn(c.dt, v.y, __fmaf_rn(c.dt_lo, v.y, u.y));
    u.z = __fmaf_rn(c.dt, v.z, __fmaf_rn(c.dt_lo, v.z, u.z));
}

// Contact modes of a mass in one step (kSlipHeld: slipping with the kinetic friction saturated at
// the horizontal force it opposes).
enum : unsigned { kFree = 0u, kStick = 1u, kSlip = 2u, kSlipHeld = 3u };

// Gravity, ground contact with static / kinetic friction, and the semi-implicit Euler update of
// one mass, given the summed spring force F.  Returns the contact mode.
//   below the ground (z = z0 + uz < 0): normal force F_n = k_g (-z) added to F_z (and the ground
//   dashpot -c_g v_z of the paper's preset); with
//   F_h = (F_x, F_y): stick (|F_h| <= mu_s F_n) zeroes F_h and the horizontal velocity, slip
//   removes mu_k F_n along F_h but never more than |F_h| (with Table II's mu_s = 0.6 < mu_k = 1.0
//   a full kinetic term could reverse F_h; when mu_k F_n >= |F_h| the horizontal force is
//   cancelled and the velocity kept);
//   v <- c (v + dt F / m), u <- u + dt v.
__device__ __forceinline__ unsigned mass_update(float4& u, float4& v, float Fx, float Fy, float Fz,
                                                const StepConst& c)
{
    unsigned mode = kFree;
    Fz = __fsub_rn(__fsub_rn(Fz, c.weight), c.weight_lo);
    const float z = __fadd_rn(u.w, u.z);
    if (c.ground_on && z < 0.f) {
        const float fn = __fmul_rn(c.k_ground, -z);
        Fz = __fadd_rn(Fz, fn);
        if (c.ground_c > 0.f) Fz = __fsub_rn(Fz, __fmul_rn(c.ground_c, v.z));   // ground dashpot
        const float fh = __fsqrt_rn(__fmaf_rn(Fy, Fy, __fmul_rn(Fx, Fx)));
        if (fh <= __fmul_rn(c.mu_s, fn)) {
            mode = kStick;
            Fx = 0.f; Fy = 0.f; v.x = 0.f; v.y = 0.f;
        } else {
            const float r = __fdiv_rn(__fmaf_rn(c.mu_k, fn, __fmul_rn(c.mu_k_lo, fn)), fh);
            if (r >= 1.0f) {
                mode = kSlipHeld;
                Fx = 0.f; Fy = 0.f;
            } else {
                mode = kSlip;
                const float s = __fsub_rn(1.0f, r);
                Fx = __fmul_rn(Fx, s);
                Fy = __fmul_rn(Fy, s);
            }
        }
    }
    integrate(u, v, Fx, Fy, Fz, c);
    return mode;
}

// mass_update with the contact mode given from outside (forced >= 0: one of kFree, kStick,
// kSlip, kSlipHeld; forced < 0: decided from the state as in mass_update).  A given mode is
// applied whatever the state: free adds no ground force; the three contact modes add
// F_n = k_g (-z) whatever the sign of z, then zero the horizontal force and velocity (stick),
// remove mu_k F_n along F_h (slip, no saturation) or zero the horizontal force (saturated slip).
// This differentiates the step map along another run's contact decisions (those of the FP64
// oracle).  Each mode's arithmetic is mass_update's, so imposing a run's own modes repeats it bit
// for bit.
__device__ __forceinline__ unsigned mass_update_imposed(float4& u, float4& v, float Fx, float Fy, float Fz,
                                                        const StepConst& c, int forced)
{
    if (forced < 0) return mass_update(u, v, Fx, Fy, Fz, c);
    Fz = __fsub_rn(__fsub_rn(Fz, c.weight), c.weight_lo);
    if (forced != (int)kFree) {
        const float z = __fadd_rn(u.w, u.z);
        const float fn = __fmul_rn(c.k_ground, -z);
        Fz = __fadd_rn(Fz, fn);
        if (c.ground_c > 0.f) Fz = __fsub_rn(Fz, __fmul_rn(c.ground_c, v.z));
        if (forced == (int)kStick) {
            Fx = 0.f; Fy = 0.f; v.x = 0.f; v.y = 0.f;
        } else if (forced == (int)kSlipHeld) {
            Fx = 0.f; Fy = 0.f;
        } else {
            const float fh = __fsqrt_rn(__fmaf_rn(Fy, Fy, __fmul_rn(Fx, Fx)));
            const float s = __fsub_rn(1.0f, __fdiv_rn(__fmaf_rn(c.mu_k, fn, __fmul_rn(c.mu_k_lo, fn)), fh));
            Fx = __fmul_rn(Fx, s);
            Fy = __fmul_rn(Fy, s);
        }
    }
    integrate(u, v, Fx, Fy, Fz, c);
    return (unsigned)forced;
}

}  // namespace vx
