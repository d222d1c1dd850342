// Reverse-mode adjoint of the lattice time stepping: the gradient of sum_r dL_df[r] * fitness_r
// with respect to the per-voxel material weight w, stiffness kappa and actuation phase phi
// (k_v = w_v kappa_v, actuation a_v sin(w t + phi_v) with a_v = w_v amp[material]).
//
// For each checkpoint segment, last to first, the host launches
//   the replay: the forward lattice kernel in recording mode from the segment's checkpoint (the
//     same code as the forward run, so every state and contact mode is reproduced bit for bit),
//     writing each step's state before the update, contact mode and horizontal force before
//     contact to device memory;
//   the reverse sweep (this kernel): one thread group per robot, one thread per grid corner,
//     the transpose of each recorded step, last to first, with the contact modes held fixed
//     (their switches are measure-zero events where the step is not differentiable).  Per step:
//       mass part: (lambda_u, lambda_v) of step n+1 -> the adjoint force lambda_F and the velocity
//         adjoint of step n;
//       spring part: each forward spring's owner forms its transpose from both endpoints'
//         recorded positions and adjoint forces, keeps its own share, accumulates the spring's
//         sensitivities to k, alpha L0 and beta L0 in registers and leaves the other endpoint's
//         share in a shared-memory plane, which that endpoint adds in direction order.
// When the forward run kept every step's record (whole-trajectory records), nothing is replayed
// and a single launch sweeps the whole run.
// The adjoints and sensitivity sums are carried from one segment's launch to the next in device
// memory; the last launch scatters the sums onto the voxels with atomics (one add per spring
// and incident voxel).
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

// Asynchronous global -> shared copy of 16 or 8 bytes (cp.async), its commit and its wait.
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes_pow)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    if (bytes_pow == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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
            // slot of this group: recorded u, adjoint force, 13 planes of spring adjoints
            float4* su = sm4 + (size_t)group * kLatticeSlotVec4 * S;
            float4* sg = su + S;
            float4* sl = sg + S;                          // plane d: lambda_d of spring (c, d)
            const int cidx = lt;
            const bool in = cidx < C;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            const bool mass = (fl >> 31) & 1u;
            const int64_t o = mo + cidx;
            const float* prm = a.prm + 39 * mo;
            float* __restrict__ accg = a.acc + 39 * mo;
            // adjoints and sensitivity sums carried over from the later segment (or their
            // initial values: the fitness is the mean of u_x over the masses)
            float lux = 0.f, luy = 0.f, luz = 0.f, lvx = 0.f, lvy = 0.f, lvz = 0.f;
            float acck[13], acca[13], accb[13];
            if (a.first) {
                if (mass) lux = (float)(a.dL_df[r] / (double)a.pv.n_mass[r]);
#pragma unroll
                for (int d = 0; d < 13; ++d) { acck[d] = 0.f; acca[d] = 0.f; accb[d] = 0.f; }
            } else {
                if (in) {
                    const float4 lu = a.lu[o], lv = a.lv[o];
                    lux = lu.x; luy = lu.y; luz = lu.z; lvx = lv.x; lvy = lv.y; lvz = lv.z;
                }
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    const bool has = (fl >> d) & 1u;
                    acck[d] = has ? accg[d * C + cidx] : 0.f;
                    acca[d] = has ? accg[(13 + d) * C + cidx] : 0.f;
                    accb[d] = has ? accg[(26 + d) * C + cidx] : 0.f;
                });
            }
            const float z0 = in ? a.u0[o].w : 0.f;
            // each step's record is copied into shared memory one step ahead (cp.async), so its
            // load latency overlaps the previous step
            float4* stage_u = sm4 + (size_t)kLatticeSlotVec4 * kBlock;           // [2][kBlock]
            float2* stage_f = reinterpret_cast<float2*>(stage_u + 2 * kBlock);   // [2][kBlock]
            int sb = 0;
            if (in) {
                const int64_t ro = (int64_t)(a.n1 - 1 - a.n0) * a.rec_stride + o;
                cp_async(&stage_u[tid], &a.rec_u[ro], 16);
                cp_async(&stage_f[tid], &a.rec_f[ro], 8);
            }
            cp_async_commit();
            for (int n = a.n1 - 1; n >= a.n0; --n) {
                cp_async_wait_all();
                float4 un = make_float4(0.f, 0.f, 0.f, 0.f);
                float2 fh = make_float2(0.f, 0.f);
                if (in) {
                    un = stage_u[sb * kBlock + tid];
                    fh = stage_f[sb * kBlock + tid];
                    if (n > a.n0) {
                        const int64_t ro = (int64_t)(n - 1 - a.n0) * a.rec_stride + o;
                        cp_async(&stage_u[(sb ^ 1) * kBlock + tid], &a.rec_u[ro], 16);
                        cp_async(&stage_f[(sb ^ 1) * kBlock + tid], &a.rec_f[ro], 8);
                    }
                }
                cp_async_commit();
                sb ^= 1;
                // mass part: (lambda_u, lambda_v) of step n+1 -> lambda_F and lambda_v of step n
                float lFx = 0.f, lFy = 0.f, lFz = 0.f;
                if (mass) mass_adjoint(__float_as_uint(un.w), z0 + un.z, fh, lux, luy, luz, lvx, lvy, lvz, lFx, lFy, lFz, c);
                if (in) {
                    su[cidx] = un;
                    sg[cidx] = make_float4(lFx, lFy, lFz, 0.f);
                }
                group_sync(bar, gthreads);
                const float2 sc = a.sc[n];
                // the parameters are re-read every step (from L1/L2) rather than held in
                // registers next to the 39 sensitivity sums: an opaque copy of the pointer keeps
                // the compiler from hoisting the loads out of the step loop
                const float* p = prm;
                asm volatile("" : "+l"(p));
                // own forward springs (a = c, b = c + offset): their transposes, the share of b
                // left in plane d for b to collect.  No branch per direction (5 % faster): an
                // absent spring has k = 0 and the corner itself as far end, so its transpose is
                // exact zeros; its sums and plane entry are never read.
                if (in) for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    const bool has = (fl >> d) & 1u;
                    const int nb = has ? cidx + lattice_offset<d>(X, XY) : cidx;
                    const float4 ub = su[nb], gb = sg[nb];
                    const float k = p[d * C + cidx];
                    const SpringEval e = spring_eval_dir<d>(
                        __fsub_rn(ub.x, un.x), __fsub_rn(ub.y, un.y), __fsub_rn(ub.z, un.z), c.edge,
                        lattice_rest<d>(c), lattice_rest_sq<d>(c), k, p[(13 + d) * C + cidx],
                        p[(26 + d) * C + cidx], sc.x, sc.y);
                    float ldx, ldy, ldz, dk, da, db;
                    spring_adjoint(e, k, lFx - gb.x, lFy - gb.y, lFz - gb.z, sc.x, sc.y, ldx, ldy, ldz, dk, da, db);
                    lux -= ldx; luy -= ldy; luz -= ldz;
                    acck[d] += dk; acca[d] += da; accb[d] += db;
                    sl[d * S + cidx] = make_float4(ldx, ldy, ldz, 0.f);
                });
                group_sync(bar, gthreads);
                // backward springs (a = c - offset, b = c): their share, computed by a
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> (16 + d)) & 1u)) return;
                    const float4 ld = sl[d * S + cidx - lattice_offset<d>(X, XY)];
                    lux += ld.x; luy += ld.y; luz += ld.z;
                });
            }
            if (!a.last) {                                // carry over to the earlier segment
                if (in) {
                    a.lu[o] = make_float4(lux, luy, luz, 0.f);
                    a.lv[o] = make_float4(lvx, lvy, lvz, 0.f);
                }
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> d) & 1u)) return;
                    accg[d * C + cidx] = acck[d];
                    accg[(13 + d) * C + cidx] = acca[d];
                    accg[(26 + d) * C + cidx] = accb[d];
                });
            } else if (in) {
                // ---- per-spring sensitivities -> per-voxel sums (mean over the incident voxels) ----
                const int64_t vo = a.pv.voff[r];
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> d) & 1u)) return;
                    spring_sens_to_voxels<d>(cidx, X, XY, nx, ny, nz, a.mat + vo, acck[d], acca[d], accb[d], c,
                                             a.g_k + vo, a.g_a + vo, a.g_b + vo);
                });
            }
            group_sync(bar, gthreads);                    // the slot is free for the next item
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
