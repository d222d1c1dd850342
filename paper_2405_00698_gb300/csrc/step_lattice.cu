// Lattice-gather time stepping: the deterministic, atomic-free resident path (Section II-C:
// spring updates then mass updates each step; Table II constants).
//
// A robot's masses sit on the corners of its voxel grid, and every spring joins a corner to one
// of its 13 "forward" lattice neighbours (offset d with a larger corner id).  Each thread owns
// one corner for the whole call and keeps in registers its displacement u, velocity v and the
// (k, alpha L0, beta L0) of its up-to-13 forward springs.  Per step:
//   phase A: for each forward spring (c, c + off(d)) the owner computes the force f from its own
//            u and the neighbour's u (shared memory), adds f to its own total and writes -f to
//            the force plane d of shared memory at index c;
//   phase B: each thread adds the plane-d entries at c - off(d) of its backward springs, then
//            applies gravity, ground contact with friction and the semi-implicit Euler update in
//            registers and publishes its new u.
// Two block barriers per step, no atomics, and a fixed summation order (own forward springs by
// direction, then backward springs by direction): bit-reproducible.
// Shared memory per robot slot: u as 3 float planes of C corners + 13 x 3 force planes.
// The state is the displacement from the rest lattice (rest height z0 in u.w), so a spring
// vector is d0 + (u_b - u_a) with d0 the exact lattice offset and the extension is formed without
// cancellation: l - L0 = (2 d0.du + du.du) / (l + L0).
#include "common.cuh"

namespace vx {
namespace {

constexpr int kMaxLatticeThreads = 768;

__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__global__ void __launch_bounds__(kMaxLatticeThreads, 1) k_step_lattice(LatticeArgs a)
{
    extern __shared__ __align__(16) float sm[];
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
        __syncthreads();   // everyone has read the item before thread 0 may overwrite it
        if (group < count) {
            const int r = a.item_robots[first + group];
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
            const int X = nx + 1, XY = (nx + 1) * (ny + 1), C = XY * (nz + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            // shared-memory slot of this group (gthreads corners): u planes then 13 x 3 force planes
            const int sc_n = gthreads;
            float* slot = sm + (size_t)group * kLatticeSlotFloats * sc_n;
            float* sx = slot;
            float* sy = sx + sc_n;
            float* sz = sy + sc_n;
            float* fb = sz + sc_n;   // plane (3d + axis) at fb + (3d + axis) * sc_n
            const int cidx = lt;
            const bool in = cidx < C;
            uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            float pk[13], pa[13], pb[13];
            const float* prm = a.prm + 39 * mo;
#pragma unroll
            for (int d = 0; d < 13; ++d) {
                const bool has = (fl >> d) & 1u;
                pk[d] = has ? prm[(0 * 13 + d) * C + cidx] : 0.f;
                pa[d] = has ? prm[(1 * 13 + d) * C + cidx] : 0.f;
                pb[d] = has ? prm[(2 * 13 + d) * C + cidx] : 0.f;
            }
            float4 u = in ? a.u[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v = in ? a.v[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            const bool mass = (fl >> 31) & 1u;
            if (in) { sx[cidx] = u.x; sy[cidx] = u.y; sz[cidx] = u.z; }
            group_sync(bar, gthreads);
            for (int n = 0; n < a.nsteps; ++n) {
                const float2 sc = a.sc[n];
                float Fx = 0.f, Fy = 0.f, Fz = 0.f;
                // phase A: forward springs
#pragma unroll
                for (int d = 0; d < 13; ++d) {
                    if (!((fl >> d) & 1u)) continue;
                    const int ox = lattice_dir(d, 0), oy = lattice_dir(d, 1), oz = lattice_dir(d, 2);
                    const int nb = cidx + ox + X * oy + XY * oz;
                    const float dux = sx[nb] - u.x, duy = sy[nb] - u.y, duz = sz[nb] - u.z;
                    const float d0x = c.edge * ox, d0y = c.edge * oy, d0z = c.edge * oz;
                    const int cls = (ox != 0) + (oy != 0) + (oz != 0);
                    const float L0 = cls == 1 ? c.edge : (cls == 2 ? c.edge_sqrt2 : c.edge_sqrt3);
                    const float dx = d0x + dux, dy = d0y + duy, dz = d0z + duz;
                    const float l2 = dx * dx + dy * dy + dz * dz;
                    const float inv = rsqrtf(l2);
                    const float l = l2 * inv;
                    const float num = 2.0f * (d0x * dux + d0y * duy + d0z * duz) + (dux * dux + duy * duy + duz * duz);
                    const float ext = __fdividef(num, l + L0) - (pa[d] * sc.x + pb[d] * sc.y);
                    const float f = l2 > 1e-30f ? pk[d] * ext * inv : 0.f;
                    const float gx = f * dx, gy = f * dy, gz = f * dz;
                    Fx += gx; Fy += gy; Fz += gz;
                    fb[(3 * d + 0) * sc_n + cidx] = -gx;
                    fb[(3 * d + 1) * sc_n + cidx] = -gy;
                    fb[(3 * d + 2) * sc_n + cidx] = -gz;
                }
                group_sync(bar, gthreads);
                // phase B: backward springs, then the mass update
#pragma unroll
                for (int d = 0; d < 13; ++d) {
                    if (!((fl >> (16 + d)) & 1u)) continue;
                    const int nb = cidx - (lattice_dir(d, 0) + X * lattice_dir(d, 1) + XY * lattice_dir(d, 2));
                    Fx += fb[(3 * d + 0) * sc_n + nb];
                    Fy += fb[(3 * d + 1) * sc_n + nb];
                    Fz += fb[(3 * d + 2) * sc_n + nb];
                }
                if (mass) {
                    Fz -= c.weight;
                    const float z = u.w + u.z;
                    if (c.ground_on && z < 0.f) {
                        const float fn = c.k_ground * (-z);
                        Fz += fn;
                        const float fh = sqrtf(Fx * Fx + Fy * Fy);
                        if (fh <= c.mu_s * fn) {
                            Fx = 0.f; Fy = 0.f; v.x = 0.f; v.y = 0.f;
                        } else {
                            const float s2 = 1.0f - c.mu_k * fn / fh;
                            Fx *= s2; Fy *= s2;
                        }
                    }
                    v.x = c.damping * (v.x + c.dt_over_m * Fx);
                    v.y = c.damping * (v.y + c.dt_over_m * Fy);
                    v.z = c.damping * (v.z + c.dt_over_m * Fz);
                    u.x += c.dt * v.x; u.y += c.dt * v.y; u.z += c.dt * v.z;
                    sx[cidx] = u.x; sy[cidx] = u.y; sz[cidx] = u.z;
                }
                group_sync(bar, gthreads);
            }
            if (in) {
                a.u[mo + cidx] = u;
                a.v[mo + cidx] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace

int lattice_max_threads() { return kMaxLatticeThreads; }

cudaError_t launch_step_lattice(const LatticeArgs& a, int grid, int threads, size_t smem,
                                cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_step_lattice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_step_lattice<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vx
