// Reverse-mode adjoint of the lattice time stepping: the gradient of sum_r dL_df[r] * fitness_r
// with respect to the per-voxel material weight w, stiffness kappa and actuation phase phi
// (k_v = w_v kappa_v, actuation a_v sin(w t + phi_v) with a_v = w_v amp[material]).
//
// One thread group per robot, one thread per grid corner, as in the forward lattice kernel.
// For each checkpoint segment, last to first:
//   replay:  the forward steps of the segment from its checkpoint with the same shared
//            arithmetic (physics.cuh) and summation order as the forward run, so every state and
//            contact mode is reproduced bit for bit; each step records the state before the
//            update, the contact mode and the horizontal force before contact;
//   reverse: the transpose of each recorded step, last to first, with the contact modes held
//            fixed (their switches are measure-zero events where the step is not differentiable):
//            the mass part turns (lambda_u, lambda_v) of step n+1 into the adjoint force
//            lambda_F and the velocity adjoint of step n; the spring part turns lambda_F into
//            lambda_u contributions and accumulates each spring's sensitivity to k, alpha L0 and
//            beta L0.
// Shared memory per robot slot: the spring parameters (read by both endpoints), u and lambda_F
// as planes over the slot's corners.  Each endpoint recomputes the springs it shares, so nothing
// is added atomically inside a robot; per-voxel gradients are accumulated with atomics at the
// end (one add per spring and incident voxel).
#include <cmath>

#include "adjoint.cuh"
#include "common.cuh"
#include "physics.cuh"

namespace vx {
namespace {

constexpr int kBlock = 768;

__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__global__ void __launch_bounds__(kBlock, 1) k_adjoint_lattice(AdjointArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    __shared__ int sh_item[4];
    const int tid = threadIdx.x;
    const StepConst c = a.c;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(a.queue, 1);
            if (it < a.n_items) {
                const int4 item = a.items[it];
                sh_item[0] = item.x; sh_item[1] = item.y; sh_item[2] = item.z; sh_item[3] = 1;
            } else {
                sh_item[3] = 0;
            }
        }
        __syncthreads();
        if (!sh_item[3]) break;
        const int first = sh_item[0], count = sh_item[1], gthreads = sh_item[2];
        const int group = tid / gthreads, lt = tid % gthreads;
        __syncthreads();
        if (group < count) {
            const int r = a.item_robots[first + group];
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
            const int X = nx + 1, XY = (nx + 1) * (ny + 1), C = XY * (nz + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            const int S = gthreads;                       // plane stride of this slot
            // slot of this group: u (float4), lambda_F (float4), 39 parameter floats per corner
            float4* su = reinterpret_cast<float4*>(reinterpret_cast<char*>(sm4) +
                                                   (size_t)group * sizeof(float) * kAdjointSlotFloats * S);
            float4* sg = su + S;                                       // lambda_F at step n
            float* prm = reinterpret_cast<float*>(sg + S);             // [3][13][S] parameters
            const int cidx = lt;
            const bool in = cidx < C;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            const bool mass = (fl >> 31) & 1u;
            if (in) {
                const float* gp = a.prm + 39 * mo;
                for (int q = 0; q < 39; ++q) prm[q * S + cidx] = gp[q * C + cidx];
            }
            const int M = a.pv.n_mass[r];
            // adjoint of the final state: the fitness is the mean of u_x over the masses
            float lux = mass ? (float)(a.dL_df[r] / (double)M) : 0.f, luy = 0.f, luz = 0.f;
            float lvx = 0.f, lvy = 0.f, lvz = 0.f;
            float acck[13], acca[13], accb[13];
#pragma unroll
            for (int d = 0; d < 13; ++d) { acck[d] = 0.f; acca[d] = 0.f; accb[d] = 0.f; }
            float4* rec_u = a.rec_u + (size_t)blockIdx.x * a.K * kBlock + (size_t)group * S;
            float2* rec_f = a.rec_f + (size_t)blockIdx.x * a.K * kBlock + (size_t)group * S;
            const float z0 = in ? a.ckpt_u[mo + cidx].w : 0.f;
            const int nseg = (a.nsteps + a.K - 1) / a.K;
            group_sync(bar, gthreads);
            for (int seg = nseg - 1; seg >= 0; --seg) {
                const int n0 = seg * a.K, n1 = min(a.nsteps, n0 + a.K);
                // ---- replay the segment from its checkpoint, recording every step ----
                float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
                if (in) {
                    const int64_t o = (int64_t)seg * a.ckpt_stride + mo + cidx;
                    u = a.ckpt_u[o];
                    v = a.ckpt_v[o];
                }
                for (int n = n0; n < n1; ++n) {
                    if (in) su[cidx] = u;
                    group_sync(bar, gthreads);
                    const float2 sc = a.sc[n];
                    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
                    for_each_dir([&](auto t) {        // own forward springs
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> d) & 1u)) return;
                        const float4 ub = su[cidx + lattice_offset<d>(X, XY)];
                        const SpringEval e = spring_eval_dir<d>(
                            __fsub_rn(ub.x, u.x), __fsub_rn(ub.y, u.y), __fsub_rn(ub.z, u.z), c.edge,
                            lattice_rest<d>(c), lattice_rest_sq<d>(c), prm[d * S + cidx], prm[(13 + d) * S + cidx],
                            prm[(26 + d) * S + cidx], sc.x, sc.y);
                        Fx = __fadd_rn(Fx, e.gx); Fy = __fadd_rn(Fy, e.gy); Fz = __fadd_rn(Fz, e.gz);
                    });
                    for_each_dir([&](auto t) {        // backward springs: the forward run's values
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> (16 + d)) & 1u)) return;
                        const int na = cidx - lattice_offset<d>(X, XY);
                        const float4 ua = su[na];
                        const SpringEval e = spring_eval_dir<d>(
                            __fsub_rn(u.x, ua.x), __fsub_rn(u.y, ua.y), __fsub_rn(u.z, ua.z), c.edge,
                            lattice_rest<d>(c), lattice_rest_sq<d>(c), prm[d * S + na], prm[(13 + d) * S + na],
                            prm[(26 + d) * S + na], sc.x, sc.y);
                        Fx = __fadd_rn(Fx, -e.gx); Fy = __fadd_rn(Fy, -e.gy); Fz = __fadd_rn(Fz, -e.gz);
                    });
                    unsigned mode = kFree;
                    const float4 ub4 = u;
                    if (mass) mode = mass_update(u, v, Fx, Fy, Fz, c);
                    if (in) {
                        rec_u[(size_t)(n - n0) * kBlock + cidx] = make_float4(ub4.x, ub4.y, ub4.z, __uint_as_float(mode));
                        rec_f[(size_t)(n - n0) * kBlock + cidx] = make_float2(Fx, Fy);
                    }
                    group_sync(bar, gthreads);
                }
                // ---- reverse sweep of the segment ----
                for (int n = n1 - 1; n >= n0; --n) {
                    float4 un = make_float4(0.f, 0.f, 0.f, 0.f);
                    float2 fh = make_float2(0.f, 0.f);
                    if (in) {
                        un = rec_u[(size_t)(n - n0) * kBlock + cidx];
                        fh = rec_f[(size_t)(n - n0) * kBlock + cidx];
                    }
                    const unsigned mode = __float_as_uint(un.w);
                    float lFx = 0.f, lFy = 0.f, lFz = 0.f;
                    if (mass) mass_adjoint(mode, z0 + un.z, fh, lux, luy, luz, lvx, lvy, lvz, lFx, lFy, lFz, c);
                    if (in) {
                        su[cidx] = un;
                        sg[cidx] = make_float4(lFx, lFy, lFz, 0.f);
                    }
                    group_sync(bar, gthreads);
                    const float2 sc = a.sc[n];
                    for_each_dir([&](auto t) {        // own forward springs: a = c, b = c + offset
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> d) & 1u)) return;
                        const int nb = cidx + lattice_offset<d>(X, XY);
                        const float4 ub = su[nb], gb = sg[nb];
                        const float k = prm[d * S + cidx];
                        const SpringEval e = spring_eval_dir<d>(
                            __fsub_rn(ub.x, un.x), __fsub_rn(ub.y, un.y), __fsub_rn(ub.z, un.z), c.edge,
                            lattice_rest<d>(c), lattice_rest_sq<d>(c), k, prm[(13 + d) * S + cidx], prm[(26 + d) * S + cidx],
                            sc.x, sc.y);
                        float ldx, ldy, ldz, dk, da, db;
                        spring_adjoint(e, k, lFx - gb.x, lFy - gb.y, lFz - gb.z, sc.x, sc.y, ldx, ldy, ldz,
                                       dk, da, db);
                        lux -= ldx; luy -= ldy; luz -= ldz;
                        acck[d] += dk; acca[d] += da; accb[d] += db;
                    });
                    for_each_dir([&](auto t) {        // backward springs: a = c - offset, b = c
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> (16 + d)) & 1u)) return;
                        const int na = cidx - lattice_offset<d>(X, XY);
                        const float4 ua = su[na], ga = sg[na];
                        const float k = prm[d * S + na];
                        const SpringEval e = spring_eval_dir<d>(
                            __fsub_rn(un.x, ua.x), __fsub_rn(un.y, ua.y), __fsub_rn(un.z, ua.z), c.edge,
                            lattice_rest<d>(c), lattice_rest_sq<d>(c), k, prm[(13 + d) * S + na], prm[(26 + d) * S + na], sc.x,
                            sc.y);
                        float ldx, ldy, ldz, dk, da, db;
                        spring_adjoint(e, k, ga.x - lFx, ga.y - lFy, ga.z - lFz, sc.x, sc.y, ldx, ldy, ldz,
                                       dk, da, db);
                        lux += ldx; luy += ldy; luz += ldz;
                    });
                    group_sync(bar, gthreads);
                }
            }
            // ---- per-spring sensitivities -> per-voxel sums (mean over the incident voxels) ----
            if (in) {
                const int64_t vo = a.pv.voff[r];
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> d) & 1u)) return;
                    spring_sens_to_voxels<d>(cidx, X, XY, nx, ny, nz, a.mat + vo, acck[d], acca[d], accb[d], c,
                                             a.g_k + vo, a.g_a + vo, a.g_b + vo);
                });
            }
        }
        __syncthreads();
    }
}

// dL/dw, dL/dkappa, dL/dphi per voxel from dL/dk_v, dL/dalpha_v, dL/dbeta_v:
//   k_v = w kappa, alpha_v = w A cos(phi), beta_v = w A sin(phi), A = amp[material].
__global__ void k_adjoint_voxels(const uint8_t* __restrict__ mat, const float* __restrict__ w,
                                 const float* __restrict__ kappa, const float* __restrict__ phi,
                                 MatConst mc, const float* __restrict__ gk, const float* __restrict__ ga,
                                 const float* __restrict__ gb, int64_t n, float* __restrict__ g_w,
                                 float* __restrict__ g_kappa, float* __restrict__ g_phi)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = mat[i];
        if (m == 0) { g_w[i] = 0.f; g_kappa[i] = 0.f; g_phi[i] = 0.f; continue; }
        const float A = mc.amp[m];
        float s, co;
        sincosf(phi[i], &s, &co);
        g_w[i] = kappa[i] * gk[i] + A * (co * ga[i] + s * gb[i]);
        g_kappa[i] = w[i] * gk[i];
        g_phi[i] = w[i] * A * (-s * ga[i] + co * gb[i]);
    }
}

}  // namespace

cudaError_t launch_adjoint_lattice(const AdjointArgs& a, int grid, int threads, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_lattice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_adjoint_lattice<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_voxels(const uint8_t* mat, const float* w, const float* kappa, const float* phi,
                                  MatConst mc, const float* g_k, const float* g_a, const float* g_b, int64_t n,
                                  float* g_w, float* g_kappa, float* g_phi, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 65535);
    k_adjoint_voxels<<<blocks, 256, 0, s>>>(mat, w, kappa, phi, mc, g_k, g_a, g_b, n, g_w, g_kappa, g_phi);
    return cudaGetLastError();
}

}  // namespace vx
