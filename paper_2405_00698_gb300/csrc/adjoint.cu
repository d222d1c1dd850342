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
//         sensitivities to k, alpha L0 and beta L0 in tensor memory and leaves the other
//         endpoint's share in a shared-memory plane, which that endpoint adds in direction order.
// When the forward run kept every step's record (whole-trajectory records), nothing is replayed
// and a single launch sweeps the whole run.
// The adjoints and sensitivity sums are carried from one segment's launch to the next in device
// memory; the last launch scatters the sums onto the voxels with atomics (one add per spring
// and incident voxel).
#include <cmath>

#include "adjoint.cuh"
#include "common.cuh"
#include "physics.cuh"
#include "tmem.cuh"

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

// Tensor-memory cells of direction D within a thread's 80 columns: (k, alpha L0) at cells_p and
// (beta L0, sum dL/dk, sum dL/d(alpha L0), sum dL/d(beta L0)) at cells_s, each pair or quad on a
// boundary of its own size.
template <int D>
__host__ __device__ constexpr uint32_t cells_p() { return D % 2 == 0 ? 6 * D + 4 : 6 * D; }
template <int D>
__host__ __device__ constexpr uint32_t cells_s() { return D % 2 == 0 ? 6 * D : 6 * D + 2; }
template <int D>
__device__ __forceinline__ void cells_load(uint32_t tm, uint32_t (&v)[6])
{
    tmem_ld2(tm + cells_p<D>(), v[0], v[1]);
    tmem_ld4(tm + cells_s<D>(), v[2], v[3], v[4], v[5]);
}

// One block of 768 threads per SM, persistent over the work items.  Each thread's 13 spring
// parameter triplets and 13 sensitivity triplets (78 floats) live in tensor memory, which the
// sweep does not otherwise use: per direction one 2-column and one 4-column load just before the
// transpose and one 4-column store of the updated sums after it.  Held in registers next to the
// sweep's other state they spilled to local memory, which misses L1 beside 221 KB of shared
// memory: 1.5x the time of this version.
// CUBE8: every item is one 8 x 8 x 8 robot in a 768-thread slot; strides and plane stride are
// compile-time constants (immediate shared-memory offsets), as in the forward kernel.
template <bool CUBE8>
__global__ void __launch_bounds__(kBlock, 1) k_adjoint_lattice(AdjointArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    __shared__ int sh_item[4];
    __shared__ uint32_t sh_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc_warp(&sh_tmem);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tm = tmem_warp_base(sh_tmem, warp);
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
        const int group = CUBE8 ? 0 : tid / gthreads, lt = CUBE8 ? tid : tid % gthreads;
        __syncthreads();
        if (group < count) {                              // whole warps (slots are multiples of 32)
            const int r = a.item_robots[first + group];
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
            const int X = CUBE8 ? 9 : nx + 1, XY = CUBE8 ? 81 : (nx + 1) * (ny + 1), C = CUBE8 ? 729 : XY * (nz + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            const int S = CUBE8 ? kBlock : gthreads;
            float4* su = sm4 + (size_t)group * kLatticeSlotVec4 * S;
            float4* sg = su + S;
            float4* sl = sg + S;
            const int cidx = lt;
            const bool in = cidx < C;
            // warps past the robot's corners skip the transposes (a uniform branch, so the
            // warp-collective tensor-memory accesses stay converged)
            const bool warp_in = (lt & ~31) < C;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            const bool mass = (fl >> 31) & 1u;
            const int64_t o = mo + cidx;
            const float* prm = a.prm + 39 * mo;
            float* __restrict__ accg = a.acc + 39 * mo;
            float lux = 0.f, luy = 0.f, luz = 0.f, lvx = 0.f, lvy = 0.f, lvz = 0.f;
            if (a.first) {
                if (mass) lux = (float)(a.dL_df[r] / (double)a.pv.n_mass[r]);
            } else if (in) {
                const float4 lu = a.lu[o], lv = a.lv[o];
                lux = lu.x; luy = lu.y; luz = lu.z; lvx = lv.x; lvy = lv.y; lvz = lv.z;
            }
            // parameters and carried sums into tensor memory (absent springs: zeros)
            if (warp_in) {
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    const bool has = (fl >> d) & 1u;
                    const float k = has ? prm[d * C + cidx] : 0.f;
                    const float pa = has ? prm[(13 + d) * C + cidx] : 0.f;
                    const float pb = has ? prm[(26 + d) * C + cidx] : 0.f;
                    const bool carried = has && !a.first;
                    const float sk = carried ? accg[d * C + cidx] : 0.f;
                    const float sa = carried ? accg[(13 + d) * C + cidx] : 0.f;
                    const float sb = carried ? accg[(26 + d) * C + cidx] : 0.f;
                    __syncwarp();
                    tmem_st2(tm + cells_p<d>(), __float_as_uint(k), __float_as_uint(pa));
                    tmem_st4(tm + cells_s<d>(), __float_as_uint(pb), __float_as_uint(sk), __float_as_uint(sa),
                             __float_as_uint(sb));
                });
                tmem_wait_st();
            }
            const float z0 = in ? a.u0[o].w : 0.f;
            float4* stage_u = sm4 + (size_t)kLatticeSlotVec4 * kBlock;           // [2][kBlock]
            float2* stage_f = reinterpret_cast<float2*>(stage_u + 2 * kBlock);   // [2][kBlock]
            int sb = 0;
            if (in) {
                const int64_t ro = (int64_t)(a.n1 - 1 - a.n0) * a.rec_stride + o;
                cp_async(&stage_u[tid], &a.rec_u[ro], 16);
                cp_async(&stage_f[tid], &a.rec_f[ro], 8);
            }
            cp_async_commit();
            int Xs = X, XYs = XY, Ss = S;
            for (int n = a.n1 - 1; n >= a.n0; --n) {
                // the lattice offsets are recomputed every step rather than hoisted out of the
                // loop and spilled: an opaque copy of the strides hides their invariance
                if constexpr (!CUBE8) asm volatile("" : "+r"(Xs), "+r"(XYs), "+r"(Ss));
                // direction 0's cells, read while the mass part runs
                uint32_t cur[6];
                if (warp_in) {
                    __syncwarp();                         // converged for the collective loads
                    cells_load<0>(tm, cur);
                }
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
                float lFx = 0.f, lFy = 0.f, lFz = 0.f;
                if (mass) mass_adjoint(__float_as_uint(un.w), z0 + un.z, fh, lux, luy, luz, lvx, lvy, lvz, lFx, lFy, lFz, c);
                if (in) {
                    su[cidx] = un;
                    sg[cidx] = make_float4(lFx, lFy, lFz, 0.f);
                }
                group_sync(bar, gthreads);
                const float2 sc = a.sc[n];
                // own forward springs: as in the register version, branch-free (an absent spring
                // has k = 0 and the corner itself as far end); lanes past the corners compute on
                // their own unused rows and their results are never read
                if (warp_in) {
                    __syncwarp();
                    tmem_wait_ld6(cur);
                    for_each_dir([&](auto t) {
                        constexpr int d = decltype(t)::value;
                        if constexpr (d > 0) {
                            cells_load<d>(tm, cur);
                            tmem_wait_ld6(cur);
                        }
                        const bool has = (fl >> d) & 1u;
                        const int nb = has ? cidx + lattice_offset<d>(Xs, XYs) : cidx;
                        const float4 ub = su[nb], gb = sg[nb];
                        const float k = __uint_as_float(cur[0]);
                        const SpringEval e = spring_eval_ends<d>(ub, un, c.edge,
                            lattice_rest<d>(c), lattice_rest_sq<d>(c), k, __uint_as_float(cur[1]),
                            __uint_as_float(cur[2]), sc.x, sc.y);
                        float ldx, ldy, ldz, dk, da, db;
                        // lambda_F_a - lambda_F_b, x and y as one paired fused multiply-add
                        const float2 lf = __ffma2_rn(make_float2(gb.x, gb.y), kMinusOne2, make_float2(lFx, lFy));
                        spring_adjoint(e, k, lf.x, lf.y, lFz - gb.z, sc.x, sc.y, ldx, ldy, ldz, dk, da, db);
                        lux -= ldx; luy -= ldy; luz -= ldz;
                        sl[d * Ss + cidx] = make_float4(ldx, ldy, ldz, e.ext);
                        __syncwarp();
                        tmem_st4(tm + cells_s<d>(), cur[2], __float_as_uint(__uint_as_float(cur[3]) + dk),
                                 __float_as_uint(__uint_as_float(cur[4]) + da),
                                 __float_as_uint(__uint_as_float(cur[5]) + db));
                    });
                    tmem_wait_st();                       // the sums are read again next step
                }
                group_sync(bar, gthreads);
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> (16 + d)) & 1u)) return;
                    const float4 ld = sl[d * Ss + cidx - lattice_offset<d>(Xs, XYs)];
                    lux += ld.x; luy += ld.y; luz += ld.z;
                });
            }
            // the sums out of tensor memory: carried to the earlier segment, or (last segment)
            // scattered onto the voxels
            if (warp_in) {
                const int64_t vo = a.pv.voff[r];
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    uint32_t v6[6];
                    __syncwarp();                         // lanes reconverge after the scatter
                    cells_load<d>(tm, v6);
                    tmem_wait_ld6(v6);
                    if (!((fl >> d) & 1u)) return;
                    const float sk = __uint_as_float(v6[3]), sa = __uint_as_float(v6[4]), sbb = __uint_as_float(v6[5]);
                    if (!a.last) {
                        accg[d * C + cidx] = sk;
                        accg[(13 + d) * C + cidx] = sa;
                        accg[(26 + d) * C + cidx] = sbb;
                    } else {
                        spring_sens_to_voxels<d>(cidx, X, XY, nx, ny, nz, a.mat + vo, sk, sa, sbb, c, a.g_k + vo,
                                                 a.g_a + vo, a.g_b + vo);
                    }
                });
            }
            if (!a.last && in) {
                a.lu[o] = make_float4(lux, luy, luz, 0.f);
                a.lv[o] = make_float4(lvx, lvy, lvz, 0.f);
            }
            group_sync(bar, gthreads);                    // the slot is free for the next item
        }
        __syncthreads();
    }
    // every thread has waited for its own tensor-memory loads and stores
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc_warp(sh_tmem);
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
    auto kernel = a.cube8 ? k_adjoint_lattice<true> : k_adjoint_lattice<false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, threads, smem, s>>>(a);
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
