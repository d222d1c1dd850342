// Cluster lattice stepping for robots too large for one block but small enough for a few
// (Section II-C: the spring and mass updates of each step; Table II constants).
//
// A robot of Z corner layers is cut into q slabs of consecutive layers, one per CTA of a
// q-CTA thread-block cluster (q <= 8), each slab of at most 768 corners: thread t of CTA k owns
// corner k * L * XY + t (L layers per slab, XY corners per layer) and keeps, like the one-block
// lattice kernel, its forward springs' parameters, u and v in registers; u, v and the 13 force
// planes live in the CTA's shared memory.  Springs between two slabs join a corner of one slab's
// top layer to the next slab's bottom layer: the owner (lower corner) reads the neighbour's u
// from the next CTA's shared memory, and the upper corner reads the force from the previous
// CTA's planes, through distributed shared memory.  Two cluster barriers per step (after the
// forces, after the mass update) and the same arithmetic and summation order as the other
// stepping kernels: a robot stepped here follows the same bits as on the streamed path.
#include <cooperative_groups.h>

#include "common.cuh"
#include "physics.cuh"

namespace cg = cooperative_groups;

namespace vx {
namespace {

constexpr int kClusterThreads = 768;

template <bool DAMPED>
__global__ void __launch_bounds__(kClusterThreads, 1) k_step_cluster(ClusterArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    cg::cluster_group cl = cg::this_cluster();
    const int q = a.q;
    const int rank = (int)cl.block_rank();
    const int r = a.robots[blockIdx.x / q];
    const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
    const int X = nx + 1, XY = (nx + 1) * (ny + 1), Z = nz + 1, C = XY * Z;
    const int L = (Z + q - 1) / q;                       // layers per slab (L * XY <= 768)
    const int z0 = min(Z, rank * L), z1 = min(Z, z0 + L);
    const int c0 = z0 * XY, c1 = z1 * XY, cprev = max(0, z0 - L) * XY;
    const int64_t mo = a.pv.moff[r];
    constexpr int S = kClusterThreads;
    float4* su = sm4;                                    // u of this slab (local corner index)
    float4* sv = su + S;                                 // v (spring dashpots)
    float4* fb = sv + S;                                 // plane d: force on a of spring (a, d)
    // the neighbouring slabs' shared memory (only dereferenced across an existing boundary)
    const float4* su_next = cl.map_shared_rank(su, rank + 1 < q ? rank + 1 : rank);
    const float4* sv_next = cl.map_shared_rank(sv, rank + 1 < q ? rank + 1 : rank);
    const float4* fb_prev = cl.map_shared_rank(fb, rank > 0 ? rank - 1 : rank);
    const int t = threadIdx.x;
    const int cidx = c0 + t;
    const bool in = cidx < c1;
    const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
    const bool mass = (fl >> 31) & 1u;
    const int zc = in ? cidx / XY : -1;
    const bool top = in && zc == z1 - 1 && z1 < Z;       // forward springs with dz = 1 leave the slab
    const bool bottom = in && zc == z0 && z0 > 0;        // backward springs with dz = 1 enter it
    float pk[13], pa[13], pb[13];
    const float* prm = a.prm + 39 * mo;
    for_each_dir([&](auto tg) {
        constexpr int d = decltype(tg)::value;
        const bool has = (fl >> d) & 1u;
        pk[d] = has ? prm[(0 * 13 + d) * C + cidx] : 0.f;
        pa[d] = has ? prm[(1 * 13 + d) * C + cidx] : 0.f;
        pb[d] = has ? prm[(2 * 13 + d) * C + cidx] : 0.f;
    });
    float4 u = in ? a.u[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = in ? a.v[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (in) {
        su[t] = u;
        if (DAMPED) sv[t] = v;
    }
    cl.sync();
    for (int n = 0; n < a.nsteps; ++n) {
        const float2 sc = a.sc[n];
        float2 Fxy = make_float2(0.f, 0.f);
        float Fz = 0.f;
        // phase A: forward springs (c, c + offset(d)).  Without dashpots no branch per
        // direction: an absent spring has zero parameters and the corner's own u as far end (its
        // load predicated off), so its force is an exact zero that leaves the sums' bits
        // unchanged, as in the one-block lattice kernel
        if (in) for_each_dir([&](auto tg) {
            constexpr int d = decltype(tg)::value;
            const bool has = (fl >> d) & 1u;
            if constexpr (DAMPED) {
                if (!has) return;
            }
            const int nb = cidx + lattice_offset<d>(X, XY);
            float4 ub = u, vb = v;
            if (has) {
                if (lattice_dir(d, 2) == 1 && top) {
                    ub = su_next[nb - c1];
                    if (DAMPED) vb = sv_next[nb - c1];
                } else {
                    ub = su[nb - c0];
                    if (DAMPED) vb = sv[nb - c0];
                }
            }
            SpringEval e = spring_eval_ends<d>(ub, u, a.c.edge,
                                              lattice_rest<d>(a.c), lattice_rest_sq<d>(a.c), pk[d], pa[d], pb[d],
                                              sc.x, sc.y);
            if constexpr (DAMPED)
                spring_dashpot(e, __fsub_rn(vb.x, v.x), __fsub_rn(vb.y, v.y), __fsub_rn(vb.z, v.z), pk[d], a.c);
            Fxy = __fadd2_rn(Fxy, make_float2(e.gx, e.gy)); Fz = __fadd_rn(Fz, e.gz);
            fb[d * S + t] = make_float4(e.gx, e.gy, e.gz, e.ext);
        });
        cl.sync();
        // phase B: backward springs (c - offset(d), c), then the mass update
        for_each_dir([&](auto tg) {
            constexpr int d = decltype(tg)::value;
            if (!((fl >> (16 + d)) & 1u)) return;
            const int na = cidx - lattice_offset<d>(X, XY);
            const float4 g = (lattice_dir(d, 2) == 1 && bottom) ? fb_prev[d * S + (na - cprev)] : fb[d * S + (na - c0)];
            Fxy = __ffma2_rn(make_float2(g.x, g.y), kMinusOne2, Fxy); Fz = __fsub_rn(Fz, g.z);
        });
        if (mass) {
            mass_update(u, v, Fxy.x, Fxy.y, Fz, a.c);
            su[t] = u;
            if (DAMPED) sv[t] = v;
        }
        cl.sync();
    }
    if (in) {
        a.u[mo + cidx] = u;
        a.v[mo + cidx] = v;
    }
}

}  // namespace

int cluster_max_threads() { return kClusterThreads; }

cudaError_t launch_step_cluster(const ClusterArgs& a, int n_robots, size_t smem, cudaStream_t s)
{
    if (n_robots == 0) return cudaSuccess;
    auto kernel = a.c.damped ? k_step_cluster<true> : k_step_cluster<false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_robots * a.q), 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

}  // namespace vx
