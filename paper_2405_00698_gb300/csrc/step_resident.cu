// Resident time stepping (Section II-C: one thread per spring for the force update, one thread
// per mass for the integration; Table II constants).  One thread block owns one robot at a
// time and keeps its whole state in shared memory for every step of the call:
//   positions  float4[M]   (read by the spring phase, written by the mass phase)
//   velocities float4[M]
//   forces     float[3][M] (accumulated by the spring phase, consumed and cleared by the
//                           mass phase)
//   springs    float4[S]   when they fit (k, alpha L0, beta L0, a | b << 15 | class << 30),
//                          otherwise streamed from device memory (L2-resident) every step.
// Blocks are persistent: each pops the next robot from a work counter over a longest-first
// order, so an uneven population runs in one launch.
#include "common.cuh"

namespace vx {
namespace {

struct SmemLayout {
    float4* pos;
    float4* vel;
    float* fx;
    float* fy;
    float* fz;
    float4* spr;
};

__device__ __forceinline__ SmemLayout carve(void* base, int max_mass, int max_spring_smem)
{
    SmemLayout L;
    char* p = (char*)base;
    L.pos = (float4*)p; p += sizeof(float4) * max_mass;
    L.vel = (float4*)p; p += sizeof(float4) * max_mass;
    L.spr = (float4*)p; p += sizeof(float4) * max_spring_smem;
    L.fx = (float*)p; p += sizeof(float) * max_mass;
    L.fy = (float*)p; p += sizeof(float) * max_mass;
    L.fz = (float*)p;
    return L;
}

// Spring force on mass a (the negative acts on b): f = k (l - L) d / l with d = x_b - x_a and
// L = L0 + alpha L0 sin(w t) + beta L0 cos(w t).  Returns false for a zero-length spring.
__device__ __forceinline__ float spring_scale(float4 q, float l2, float sn, float cs,
                                              const StepConst& c)
{
    const unsigned bits = __float_as_uint(q.w);
    const unsigned cls = bits >> 30;
    const float L0 = cls == 1u ? c.edge : (cls == 2u ? c.edge_sqrt2 : c.edge_sqrt3);
    const float L = L0 + q.y * sn + q.z * cs;
    const float inv = rsqrtf(l2);
    return l2 > 1e-30f ? q.x * (1.0f - L * inv) : 0.0f;
}

__global__ void __launch_bounds__(1024, 1) k_step_resident_atomic(ResidentArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int sh_robot;
    const SmemLayout L = carve(smem_raw, a.max_mass, a.max_spring_smem);
    const int tid = threadIdx.x, T = blockDim.x;
    const StepConst c = a.c;
    int iter = 0;
    for (;;) {
        if (tid == 0) {
            int idx = a.queue ? atomicAdd(a.queue, 1) : blockIdx.x + iter * gridDim.x;
            sh_robot = idx < a.pv.P ? (a.order ? a.order[idx] : idx) : -1;
        }
        ++iter;
        __syncthreads();
        const int r = sh_robot;
        if (r < 0) break;
        const int M = a.pv.n_mass[r], S = a.pv.n_spring[r];
        const int64_t mo = a.pv.moff[r], so = a.pv.soff[r];
        for (int m = tid; m < M; m += T) {
            L.pos[m] = a.x[mo + m];
            L.vel[m] = a.v[mo + m];
            L.fx[m] = 0.f; L.fy[m] = 0.f; L.fz[m] = 0.f;
        }
        const bool spr_in_smem = S <= a.max_spring_smem;
        const float4* spr = spr_in_smem ? L.spr : a.spr_pack + so;
        if (spr_in_smem)
            for (int s = tid; s < S; s += T) L.spr[s] = a.spr_pack[so + s];
        __syncthreads();
        for (int n = 0; n < a.nsteps; ++n) {
            const float2 sc = a.sc[n];
            for (int s = tid; s < S; s += T) {
                const float4 q = spr[s];
                const unsigned bits = __float_as_uint(q.w);
                const int ia = bits & 0x7fffu, ib = (bits >> 15) & 0x7fffu;
                const float4 pa = L.pos[ia], pb = L.pos[ib];
                const float dx = pb.x - pa.x, dy = pb.y - pa.y, dz = pb.z - pa.z;
                const float l2 = dx * dx + dy * dy + dz * dz;
                const float f = spring_scale(q, l2, sc.x, sc.y, c);
                const float gx = f * dx, gy = f * dy, gz = f * dz;
                atomicAdd(&L.fx[ia], gx); atomicAdd(&L.fy[ia], gy); atomicAdd(&L.fz[ia], gz);
                atomicAdd(&L.fx[ib], -gx); atomicAdd(&L.fy[ib], -gy); atomicAdd(&L.fz[ib], -gz);
            }
            __syncthreads();
            for (int m = tid; m < M; m += T) {
                float fx = L.fx[m], fy = L.fy[m], fz = L.fz[m] - c.weight;
                L.fx[m] = 0.f; L.fy[m] = 0.f; L.fz[m] = 0.f;
                float4 x = L.pos[m], v = L.vel[m];
                if (c.ground_on && x.z < 0.f) {
                    const float fn = c.k_ground * (-x.z);
                    fz += fn;
                    const float fh = sqrtf(fx * fx + fy * fy);
                    if (fh <= c.mu_s * fn) {
                        fx = 0.f; fy = 0.f; v.x = 0.f; v.y = 0.f;
                    } else {
                        const float sc2 = 1.0f - c.mu_k * fn / fh;
                        fx *= sc2; fy *= sc2;
                    }
                }
                v.x = c.damping * (v.x + c.dt_over_m * fx);
                v.y = c.damping * (v.y + c.dt_over_m * fy);
                v.z = c.damping * (v.z + c.dt_over_m * fz);
                x.x += c.dt * v.x; x.y += c.dt * v.y; x.z += c.dt * v.z;
                L.pos[m] = x;
                L.vel[m] = v;
            }
            __syncthreads();
        }
        for (int m = tid; m < M; m += T) {
            a.x[mo + m] = L.pos[m];
            a.v[mo + m] = L.vel[m];
        }
        __syncthreads();
    }
}

}  // namespace

size_t resident_smem_bytes(int max_mass, int max_spring_smem, int accumulate)
{
    (void)accumulate;
    return sizeof(float4) * 2 * (size_t)max_mass + sizeof(float4) * (size_t)max_spring_smem +
           sizeof(float) * 3 * (size_t)max_mass;
}

cudaError_t launch_step_resident(const ResidentArgs& a, int grid, int threads, size_t smem,
                                 cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_step_resident_atomic,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_step_resident_atomic<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vx
