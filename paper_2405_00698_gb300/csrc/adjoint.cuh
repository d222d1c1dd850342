// Pieces of the reverse sweep shared by the two adjoint kernels (the resident lattice adjoint and
// the streamed one for robots too large for one SM): the transpose of the mass update with its
// contact mode held fixed, the transpose of one spring, and the scatter of a spring's summed
// sensitivities onto its incident voxels.
#pragma once

#include "common.cuh"
#include "physics.cuh"

namespace vx {

// Transpose of mass_update for a mass that took contact mode `mode` (z: its height before the
// update, fh: the horizontal spring force before contact).  On entry (lu, lv) are the adjoints of
// the state after the step; on exit lv is the adjoint of the velocity before it, lu.z has gained
// the ground-force term, and lF is the adjoint of the summed spring force.
//   v' = c (v~ + dt F~ / m), u' = u + dt v'.
__device__ __forceinline__ void mass_adjoint(unsigned mode, float z, float2 fh, float& lux, float& luy,
                                             float& luz, float& lvx, float& lvy, float& lvz, float& lFx,
                                             float& lFy, float& lFz, const StepConst& c)
{
    // the transposes of integrate(): the constants as pairs, the damping as its complement
    const float l1x = fmaf(c.dt, lux, fmaf(c.dt_lo, lux, lvx));
    const float l1y = fmaf(c.dt, luy, fmaf(c.dt_lo, luy, lvy));
    const float l1z = fmaf(c.dt, luz, fmaf(c.dt_lo, luz, lvz));
    const float tx = fmaf(-c.damping_c, l1x, l1x), ty = fmaf(-c.damping_c, l1y, l1y),
                tz = fmaf(-c.damping_c, l1z, l1z);
    const float fx = fmaf(c.dt_over_m, tx, c.dtm_lo * tx), fy = fmaf(c.dt_over_m, ty, c.dtm_lo * ty),
                fz = fmaf(c.dt_over_m, tz, c.dtm_lo * tz);
    if (mode == kFree) {
        lFx = fx; lFy = fy; lFz = fz;
        lvx = tx; lvy = ty; lvz = tz;
    } else if (mode == kStick) {
        // horizontal force and velocity were zeroed; F_n = k_g (-z) adds to F_z
        lFx = 0.f; lFy = 0.f; lFz = fz;
        lvx = 0.f; lvy = 0.f; lvz = tz;
        luz += -c.k_ground * fz;
    } else if (mode == kSlipHeld) {
        // saturated kinetic friction: the horizontal force was cancelled, the velocity kept
        lFx = 0.f; lFy = 0.f; lFz = fz;
        lvx = tx; lvy = ty; lvz = tz;
        luz += -c.k_ground * fz;
    } else {
        // slip: F~_h = F_h (1 - mu_k F_n / |F_h|), F~_z = F_z + F_n
        const float fn = c.k_ground * -z;
        const float fhm = sqrtf(fh.x * fh.x + fh.y * fh.y);
        const float hx = fh.x / fhm, hy = fh.y / fhm;
        const float rr = fmaf(c.mu_k, fn, c.mu_k_lo * fn) / fhm;
        const float ul = hx * fx + hy * fy;
        lFx = fx - rr * (fx - hx * ul);
        lFy = fy - rr * (fy - hy * ul);
        lFz = fz;
        const float lfn = -fmaf(c.mu_k, ul, c.mu_k_lo * ul) + fz;
        luz += -c.k_ground * lfn;
        lvx = tx; lvy = ty; lvz = tz;
    }
}

// Adjoint of one spring evaluated as e (force g on endpoint a), given lambda_f = lambda_F_a -
// lambda_F_b: returns lambda_d (the adjoint of d = x_b - x_a) in (ldx, ldy, ldz) and the
// sensitivities dL/dk, dL/d(alpha L0), dL/d(beta L0) of this step.
//   f = k (l - L) d / l:  df/dd = k [ (l - L)/l I + (L/l) u u^T ],  u = d / l;
//   df/dk = (l - L) u;    df/dL = -k u;   L = L0 + (alpha L0) sin + (beta L0) cos.
__device__ __forceinline__ void spring_adjoint(const SpringEval& e, float k, float lfx, float lfy,
                                               float lfz, float sn, float cs, float& ldx,
                                               float& ldy, float& ldz, float& dk, float& da,
                                               float& db)
{
    const float ul = (e.dx * lfx + e.dy * lfy + e.dz * lfz) * e.inv;    // u . lambda_f
    const float ei = e.ext * e.inv;                                      // (l - L) / l
    const float a1 = k * ei;
    const float a2 = k * (1.0f - ei) * ul * e.inv;                       // k (L/l) (u.lf) / l
    ldx = a1 * lfx + a2 * e.dx;
    ldy = a1 * lfy + a2 * e.dy;
    ldz = a1 * lfz + a2 * e.dz;
    dk = e.ext * ul;
    const float lL = -k * ul;
    da = lL * sn;
    db = lL * cs;
}

// Scatter of the summed sensitivities (to k, alpha L0, beta L0) of the forward spring along
// direction D from corner cidx onto the kept voxels around it: each gets the mean share
// (dL/dk_v += s_k / count, dL/dalpha_v += s_a L0 / count, dL/dbeta_v += s_b L0 / count), by
// atomics (a voxel receives from many springs).  mat, g_k, g_a, g_b: this robot's voxels.
template <int D>
__device__ __forceinline__ void spring_sens_to_voxels(int cidx, int X, int XY, int nx, int ny, int nz,
                                                      const uint8_t* mat, float sk, float sa, float sb,
                                                      const StepConst& c, float* g_k, float* g_a, float* g_b)
{
    const int ci = cidx % X, cj = (cidx / X) % (ny + 1), ck = cidx / XY;
    const int dd[3] = {lattice_dir(D, 0), lattice_dir(D, 1), lattice_dir(D, 2)};
    const int c0[3] = {ci, cj, ck};
    const int nn[3] = {nx, ny, nz};
    int lo[3], hi[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (dd[q] != 0) { lo[q] = hi[q] = dd[q] > 0 ? c0[q] : c0[q] - 1; }
        else { lo[q] = c0[q] - 1; hi[q] = c0[q]; }
        lo[q] = max(lo[q], 0);
        hi[q] = min(hi[q], nn[q] - 1);
    }
    int cnt = 0;
    for (int zz = lo[2]; zz <= hi[2]; ++zz)
        for (int yy = lo[1]; yy <= hi[1]; ++yy)
            for (int xx = lo[0]; xx <= hi[0]; ++xx) cnt += mat[xx + nx * (yy + ny * zz)] != 0;
    const float L0 = lattice_rest<D>(c);
    const float inv = 1.0f / (float)cnt;
    const float gk = sk * inv, ga = sa * L0 * inv, gb = sb * L0 * inv;
    for (int zz = lo[2]; zz <= hi[2]; ++zz)
        for (int yy = lo[1]; yy <= hi[1]; ++yy)
            for (int xx = lo[0]; xx <= hi[0]; ++xx) {
                const int vv = xx + nx * (yy + ny * zz);
                if (!mat[vv]) continue;
                atomicAdd(&g_k[vv], gk);
                atomicAdd(&g_a[vv], ga);
                atomicAdd(&g_b[vv], gb);
            }
}

}  // namespace vx
