// Resident time stepping (Section II-C: one thread per spring for the force update, one thread
// per mass for the integration; Table II constants).  One thread block owns one robot at a
// time and keeps its whole state in shared memory for every step of the call:
//   u       float4[C]   per grid corner: displacement from the rest lattice (ux, uy, uz) and
//                       rest height z0 (corners without a mass are carried along unchanged)
//   v       float4[C]   velocity
//   F       float[3][C] accumulated by the spring phase, consumed and cleared by the mass phase
//   springs float4[S]   (k, alpha L0, beta L0, a | b << 14 | direction << 28), ordered by
//                       direction then a, so a warp's atomic updates hit distinct masses:
//                       thread t's springs t, t + T, t + 2T, ... the first tm_rec of them in
//                       tensor memory (when the block has an SM to itself: 16 springs per thread
//                       at 1024 threads), then as many as fit in shared memory, the rest read
//                       from device memory (L2) every step.  A spring read from tensor memory
//                       takes no shared-memory bandwidth, which bounds this kernel.
// Keeping the displacement instead of the position keeps float32 precise: a spring vector is
// d = d0 + (u_b - u_a) with d0 the exact lattice offset, and the extension is formed without
// cancellation as l - L0 = (2 d0.du + du.du) / (l + L0).
// Blocks are persistent: each pops the next robot from a work counter over a longest-first
// order, so an uneven population runs in one launch.
#include "common.cuh"
#include "physics.cuh"
#include "tmem.cuh"

namespace vx {
namespace {

struct SmemLayout {
    float4* u;
    float4* vel;
    float4* spr;
    float* fx;
    float* fy;
    float* fz;
    uint32_t* massbits;
};

__device__ __forceinline__ SmemLayout carve(void* base, int max_mass, int max_spring_smem)
{
    SmemLayout L;
    char* p = (char*)base;
    L.u = (float4*)p; p += sizeof(float4) * max_mass;
    L.vel = (float4*)p; p += sizeof(float4) * max_mass;
    L.spr = (float4*)p; p += sizeof(float4) * max_spring_smem;
    L.fx = (float*)p; p += sizeof(float) * max_mass;
    L.fy = (float*)p; p += sizeof(float) * max_mass;
    L.fz = (float*)p; p += sizeof(float) * max_mass;
    L.massbits = (uint32_t*)p;
    return L;
}

__global__ void __launch_bounds__(1024, 1) k_step_resident_atomic(ResidentArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int sh_robot;
    __shared__ float4 sh_d0[13];   // lattice offset of each direction, rest length in .w
    __shared__ uint32_t sh_tmem;
    const SmemLayout L = carve(smem_raw, a.max_mass, a.max_spring_smem);
    const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5;
    const StepConst c = a.c;
    const int tm_rec = a.tm_rec;
    if (tm_rec > 0) {
        if (warp == 0) tmem_alloc_warp(&sh_tmem);
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
    }
    // this thread's cells: lane quarter warp % 4, a_tm_cols-column block per warp of the quarter
    const uint32_t tmb = tm_rec > 0 ? sh_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(a.tm_cols * (warp >> 2)) : 0u;
    if (tid < 13) {
        const int ix = lattice_dir(tid, 0), iy = lattice_dir(tid, 1), iz = lattice_dir(tid, 2);
        const float dx = c.edge * ix, dy = c.edge * iy, dz = c.edge * iz;
        const int cls = (ix != 0) + (iy != 0) + (iz != 0);
        sh_d0[tid] = make_float4(dx, dy, dz, cls == 1 ? c.edge : (cls == 2 ? c.edge_sqrt2 : c.edge_sqrt3));
    }
    int iter = 0;
    for (;;) {
        if (tid == 0) {
            int idx = a.queue ? atomicAdd(a.queue, 1) : blockIdx.x + iter * gridDim.x;
            sh_robot = idx < a.n_robots ? a.order[idx] : -1;
        }
        ++iter;
        __syncthreads();
        const int r = sh_robot;
        if (r < 0) break;
        const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
        const int M = (nx + 1) * (ny + 1) * (nz + 1);   // corners: state is indexed by corner
        const int S = a.pv.n_spring[r];
        const int64_t mo = a.pv.moff[r], so = a.pv.soff[r];
        for (int m = tid; m < M; m += T) {
            L.u[m] = a.x[mo + m];
            L.vel[m] = a.v[mo + m];
            L.fx[m] = 0.f; L.fy[m] = 0.f; L.fz[m] = 0.f;
        }
        // thread t's first springs t + j T (j < jt) in tensor memory, the next ones of the
        // direction-major list in shared memory as far as they fit, the rest read from device
        // memory (L2) every step
        const float4* __restrict__ spr_g = a.spr_pack + so;
        const int jt = min(tm_rec, (S + T - 1) / T);      // uniform over the block
        const int base = jt * T;
        const int nsm = max(0, min(S - base, a.max_spring_smem));
        for (int s = tid; s < nsm; s += T) L.spr[s] = spr_g[base + s];
        for (int j = 0; j < jt; ++j) {
            const int s = tid + j * T;
            const float4 q = s < S ? spr_g[s] : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            tmem_st4(tmb + 4 * j, __float_as_uint(q.x), __float_as_uint(q.y), __float_as_uint(q.z), __float_as_uint(q.w));
        }
        if (jt > 0) tmem_wait_st();
        // which corners carry a mass, one bit each
        for (int w = tid; w < (M + 31) / 32; w += T) {
            uint32_t bits = 0u;
            for (int b = 0; b < 32 && 32 * w + b < M; ++b)
                bits |= (a.cflags[mo + 32 * w + b] >> 31) << b;
            L.massbits[w] = bits;
        }
        __syncthreads();
        for (int n = 0; n < a.nsteps; ++n) {
            const float2 sc = a.sc[n];
            auto spring = [&](const float4 q) {
                const unsigned bits = __float_as_uint(q.w);
                const int ia = bits & 0x3fffu, ib = (bits >> 14) & 0x3fffu, dir = bits >> 28;
                const float4 ua = L.u[ia], ub = L.u[ib], d0 = sh_d0[dir];
                const float dux = ub.x - ua.x, duy = ub.y - ua.y, duz = ub.z - ua.z;
                const float dx = d0.x + dux, dy = d0.y + duy, dz = d0.z + duz;
                const float l2 = dx * dx + dy * dy + dz * dz;
                const float inv = rsqrtf(l2);
                const float l = l2 * inv;
                const float num = 2.0f * (d0.x * dux + d0.y * duy + d0.z * duz) +
                                  (dux * dux + duy * duy + duz * duz);
                const float ext = __fdividef(num, l + d0.w) - (q.y * sc.x + q.z * sc.y);
                float f = l2 > 1e-30f ? q.x * ext * inv : 0.0f;
                if (c.damped) {     // spring dashpot of the paper's preset
                    const float4 va = L.vel[ia], vb = L.vel[ib];
                    const float rv = ((vb.x - va.x) * dx + (vb.y - va.y) * dy + (vb.z - va.z) * dz) * inv;
                    f += c.spring_c * sqrtf(q.x) * rv * inv;
                }
                const float gx = f * dx, gy = f * dy, gz = f * dz;
                atomicAdd(&L.fx[ia], gx); atomicAdd(&L.fy[ia], gy); atomicAdd(&L.fz[ia], gz);
                atomicAdd(&L.fx[ib], -gx); atomicAdd(&L.fy[ib], -gy); atomicAdd(&L.fz[ib], -gz);
            };
            for (int j = 0; j < jt; ++j) {
                uint32_t r[4];
                __syncwarp();                             // converged for the collective load
                tmem_ld4(tmb + 4 * j, r[0], r[1], r[2], r[3]);
                tmem_wait_ld4(r);
                if (tid + j * T < S)
                    spring(make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]),
                                       __uint_as_float(r[3])));
            }
            for (int s = base + tid; s < S; s += T) spring(s - base < nsm ? L.spr[s - base] : spr_g[s]);
            __syncthreads();
            for (int m = tid; m < M; m += T) {
                if (!((L.massbits[m >> 5] >> (m & 31)) & 1u)) continue;   // a corner without a mass
                float fx = L.fx[m], fy = L.fy[m], fz = L.fz[m] - c.weight - c.weight_lo;
                L.fx[m] = 0.f; L.fy[m] = 0.f; L.fz[m] = 0.f;
                float4 u = L.u[m], v = L.vel[m];
                const float z = u.w + u.z;
                if (c.ground_on && z < 0.f) {
                    const float fn = c.k_ground * (-z);
                    fz += fn;
                    fz -= c.ground_c * v.z;
                    const float fh = sqrtf(fx * fx + fy * fy);
                    if (fh <= c.mu_s * fn) {
                        fx = 0.f; fy = 0.f; v.x = 0.f; v.y = 0.f;
                    } else {
                        // kinetic friction removes at most |F_h| (saturated: F_h cancelled)
                        const float r = fmaf(c.mu_k, fn, c.mu_k_lo * fn) / fh;
                        const float s2 = r >= 1.0f ? 0.0f : 1.0f - r;
                        fx *= s2; fy *= s2;
                    }
                }
                integrate(u, v, fx, fy, fz, c);
                L.u[m] = u;
                L.vel[m] = v;
            }
            __syncthreads();
        }
        for (int m = tid; m < M; m += T) {
            a.x[mo + m] = L.u[m];
            a.v[mo + m] = L.vel[m];
        }
        __syncthreads();
    }
    if (tm_rec > 0) {                              // every thread has waited for its own accesses
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (warp == 0) tmem_dealloc_warp(sh_tmem);
    }
}

}  // namespace

size_t resident_smem_bytes(int max_mass, int max_spring_smem, int accumulate)
{
    (void)accumulate;
    return sizeof(float4) * 2 * (size_t)max_mass + sizeof(float4) * (size_t)max_spring_smem +
           sizeof(float) * 3 * (size_t)max_mass + sizeof(uint32_t) * (((size_t)max_mass + 31) / 32);
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
