// Shared-memory bandwidth probe: the measured denominator of the resident kernels' roofline
// (their state lives in shared memory, so HBM does not bound them).  Every thread streams 16-byte
// loads from its block's shared memory, a warp's 32 loads covering 512 contiguous bytes (four
// 128-byte wavefronts, no bank conflicts), two 1024-thread blocks per SM; the loaded values are
// summed so that no load can be dropped.
#include "common.cuh"

namespace vx {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeVec = 2048;   // float4 per block: 32 KB
constexpr int kProbeUnroll = 8;

__global__ void __launch_bounds__(kProbeThreads) k_probe_smem(int iters, float* sink)
{
    __shared__ float4 buf[kProbeVec];
    const int t = threadIdx.x;
    for (int i = t; i < kProbeVec; i += blockDim.x) buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
    int idx = t;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k) {
            const float4 x = buf[(idx + 256 * k) & (kProbeVec - 1)];
            ax += x.x; ay += x.y; az += x.z; aw += x.w;
        }
        idx = (idx + 1) & (kProbeVec - 1);
    }
    if (ax + ay + az + aw == -1.f) sink[blockIdx.x] = ax;   // never true: keeps the sums live
}

}  // namespace

size_t probe_smem_bytes_per_iter(int grid) { return (size_t)grid * kProbeThreads * kProbeUnroll * sizeof(float4); }

cudaError_t launch_probe_smem(int grid, int iters, float* sink, cudaStream_t s)
{
    k_probe_smem<<<grid, kProbeThreads, 0, s>>>(iters, sink);
    return cudaGetLastError();
}

}  // namespace vx
