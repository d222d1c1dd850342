// The paper's own kernel organisation, kept as the measured baseline of the batched paths
// (Section II-C: each CUDA thread updates one spring or one mass of one robot): for one robot per
// launch, a spring pass (one thread per spring, force added to the endpoints' accumulators in
// device memory with atomics) and a mass pass (one thread per mass: gravity, contact, integration,
// accumulator reset).  Two launches per robot per step, state in device memory.  Same spring and
// mass arithmetic as the other paths (physics.cuh); the force sums are taken in atomic order.
#include "common.cuh"
#include "physics.cuh"

namespace vx {
namespace {

constexpr int kPlainThreads = 256;

__global__ void __launch_bounds__(kPlainThreads)
k_plain_springs(const int2* __restrict__ ab, const float4* __restrict__ prm, const int* __restrict__ mass_corner,
                const float4* __restrict__ u, const float4* __restrict__ v, float* __restrict__ F, int S, int X,
                int XY, const float2* sc_tab, int n, StepConst c)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int2 e = ab[s];
    const float4 p = prm[s];                         // (L0, k, alpha, beta)
    const int ca = mass_corner[e.x], cb = mass_corner[e.y];
    // lattice offset from the corner coordinates (exact multiples of the edge)
    const int ox = cb % X - ca % X, oy = (cb / X) % (XY / X) - (ca / X) % (XY / X), oz = cb / XY - ca / XY;
    const float4 ua = u[ca], ub = u[cb];
    const float2 sc = sc_tab[n];
    SpringEval ev = spring_eval_rt(__fsub_rn(ub.x, ua.x), __fsub_rn(ub.y, ua.y), __fsub_rn(ub.z, ua.z),
                                   ox, oy, oz, c.edge, p.x, lattice_rest_sq_rt(ox, oy, oz, c), p.y, p.z * p.x,
                                   p.w * p.x, sc.x, sc.y);
    if (c.damped) {
        const float4 va = v[ca], vb = v[cb];
        spring_dashpot(ev, __fsub_rn(vb.x, va.x), __fsub_rn(vb.y, va.y), __fsub_rn(vb.z, va.z), p.y, c);
    }
    atomicAdd(&F[3 * ca + 0], ev.gx); atomicAdd(&F[3 * ca + 1], ev.gy); atomicAdd(&F[3 * ca + 2], ev.gz);
    atomicAdd(&F[3 * cb + 0], -ev.gx); atomicAdd(&F[3 * cb + 1], -ev.gy); atomicAdd(&F[3 * cb + 2], -ev.gz);
}

__global__ void __launch_bounds__(kPlainThreads)
k_plain_masses(const int* __restrict__ mass_corner, float4* __restrict__ u, float4* __restrict__ v,
               float* __restrict__ F, int M, StepConst c)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int cc = mass_corner[m];
    float4 uu = u[cc], vv = v[cc];
    const float fx = F[3 * cc + 0], fy = F[3 * cc + 1], fz = F[3 * cc + 2];
    F[3 * cc + 0] = 0.f; F[3 * cc + 1] = 0.f; F[3 * cc + 2] = 0.f;
    mass_update(uu, vv, fx, fy, fz, c);
    u[cc] = uu;
    v[cc] = vv;
}

}  // namespace

cudaError_t launch_step_plain_robot(const int2* ab, const float4* prm, const int* mass_corner, float4* u,
                                    float4* v, float* F, int S, int M, int nx, int ny, const float2* sc, int n,
                                    StepConst c, cudaStream_t s)
{
    const int X = nx + 1, XY = (nx + 1) * (ny + 1);
    if (S > 0) k_plain_springs<<<(S + kPlainThreads - 1) / kPlainThreads, kPlainThreads, 0, s>>>(
        ab, prm, mass_corner, u, v, F, S, X, XY, sc, n, c);
    if (M > 0) k_plain_masses<<<(M + kPlainThreads - 1) / kPlainThreads, kPlainThreads, 0, s>>>(mass_corner, u, v, F, M, c);
    return cudaGetLastError();
}

}  // namespace vx
