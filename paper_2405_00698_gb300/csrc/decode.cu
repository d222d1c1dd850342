// Decoding genomes into per-voxel material, weight, stiffness and phase.
//   * direct materials / per-voxel parameters / per-voxel material scores;
//   * Gaussian positional encoding, Eq. (1), evaluated once per grid shape in FP64 and stored as
//     bfloat16 (the operand type of the tensor-core MLP);
//   * a SIMT MLP query (CUDA cores, bfloat16-rounded operands, FP32 accumulation), kept beside
//     the tensor-core kernel as the reference-speed baseline and cross-check.
#include <cuda_bf16.h>

#include "common.cuh"

namespace vx {
namespace {

__global__ void k_decode_materials(const uint8_t* __restrict__ in, int64_t n, MatConst mc,
                                   uint8_t* mat, float* w, float* kappa, float* phi, int* bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int m = in[i];
        if (m >= kNumMat) { m = 0; atomicOr(bad, 2); }
        mat[i] = (uint8_t)m;
        w[i] = 1.0f;
        kappa[i] = mc.k[m];
        phi[i] = mc.phase[m];
    }
}

__global__ void k_decode_logits(const float* __restrict__ in, int64_t n, MatConst mc,
                                uint8_t* mat, float* w, float* kappa, float* phi)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float* l = in + 5 * i;
        int best = 0;
        float bv = l[0];
#pragma unroll
        for (int c = 1; c < kNumMat; ++c)
            if (l[c] > bv) { bv = l[c]; best = c; }
        mat[i] = (uint8_t)best;
        w[i] = 1.0f;
        kappa[i] = mc.k[best];
        phi[i] = mc.phase[best];
    }
}

__global__ void k_decode_params(const uint8_t* __restrict__ mats, const float* __restrict__ w_in,
                                const float* __restrict__ k_in, const float* __restrict__ p_in,
                                int64_t n, uint8_t* mat, float* w, float* kappa, float* phi,
                                int* bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int m = mats[i];
        if (m >= kNumMat) { m = 0; atomicOr(bad, 2); }
        mat[i] = (uint8_t)m;
        w[i] = w_in[i];
        kappa[i] = k_in[i];
        phi[i] = p_in[i];
    }
}

// The same parametrisation read from genome rows [w (V) | kappa (V) | phi (V)] per robot.
__global__ void k_decode_param_rows(const uint8_t* __restrict__ mats, const float* __restrict__ rows,
                                    int64_t V, int64_t n, uint8_t* mat, float* w, float* kappa,
                                    float* phi, int* bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / V, v = i - r * V;
        const float* row = rows + 3 * V * r;
        int m = mats[i];
        if (m >= kNumMat) { m = 0; atomicOr(bad, 2); }
        mat[i] = (uint8_t)m;
        w[i] = row[v];
        kappa[i] = row[V + v];
        phi[i] = row[2 * V + v];
    }
}

// Eq. (1): gamma(v) = [cos(2 pi B v), sin(2 pi B v)], v the voxel centre normalised to [0,1]^3.
// FP64 with explicit round-to-nearest operations (no contraction), then rounded once to
// bfloat16.  One thread per (query, row of B).
__global__ void k_pe_table(int nx, int ny, int nz, const float* __restrict__ B,
                           __nv_bfloat16* __restrict__ out)
{
    const int Q = nx * ny * nz;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Q * kPeRows) return;
    const int q = idx / kPeRows, r = idx % kPeRows;
    const int i = q % nx, j = (q / nx) % ny, k = q / (nx * ny);
    const double v0 = __ddiv_rn(i + 0.5, (double)nx);
    const double v1 = __ddiv_rn(j + 0.5, (double)ny);
    const double v2 = __ddiv_rn(k + 0.5, (double)nz);
    double bv = __dmul_rn((double)B[3 * r + 0], v0);
    bv = __dadd_rn(bv, __dmul_rn((double)B[3 * r + 1], v1));
    bv = __dadd_rn(bv, __dmul_rn((double)B[3 * r + 2], v2));
    const double arg = __dmul_rn(2.0 * 3.141592653589793, bv);
    double s, c;
    sincos(arg, &s, &c);
    out[(size_t)q * kPeDim + r] = __double2bfloat16(c);
    out[(size_t)q * kPeDim + kPeRows + r] = __double2bfloat16(s);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// SIMT MLP query: one block per genome, one thread per query point at a time.  Weights are
// rounded to bfloat16 in shared memory; activations are rounded to bfloat16 between layers, as
// the tensor-core operands are.
constexpr int kSimtThreads = 128;

__global__ void __launch_bounds__(kSimtThreads)
k_mlp_simt(int Q, const __nv_bfloat16* __restrict__ pe, const float* __restrict__ genomes,
           MatConst mc, uint8_t* mat, float* w, float* kappa, float* phi)
{
    extern __shared__ float sm[];
    float* W1 = sm;                       // [64][256]
    float* W2 = W1 + kHidden * kPeDim;    // [64][64]
    float* W3 = W2 + kHidden * kHidden;   // [6][64]
    float* bias = W3 + kOut * kHidden;    // b1[64], b2[64], b3[6]
    const int g = blockIdx.x;
    const float* G = genomes + (size_t)g * kGenome;
    for (int i = threadIdx.x; i < kHidden * kPeDim; i += blockDim.x) W1[i] = bf16r(G[kOffW1 + i]);
    for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) W2[i] = bf16r(G[kOffW2 + i]);
    for (int i = threadIdx.x; i < kOut * kHidden; i += blockDim.x) W3[i] = bf16r(G[kOffW3 + i]);
    for (int i = threadIdx.x; i < kHidden; i += blockDim.x) {
        bias[i] = G[kOffB1 + i];
        bias[kHidden + i] = G[kOffB2 + i];
    }
    if (threadIdx.x < kOut) bias[2 * kHidden + threadIdx.x] = G[kOffB3 + threadIdx.x];
    __syncthreads();
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
        const __nv_bfloat16* gam = pe + (size_t)q * kPeDim;
        float h1[kHidden];
#pragma unroll
        for (int o = 0; o < kHidden; ++o) h1[o] = 0.f;
        for (int c = 0; c < kPeDim; ++c) {
            float x = __bfloat162float(gam[c]);
#pragma unroll
            for (int o = 0; o < kHidden; ++o) h1[o] = fmaf(W1[o * kPeDim + c], x, h1[o]);
        }
#pragma unroll
        for (int o = 0; o < kHidden; ++o) h1[o] = bf16r(fmaxf(h1[o] + bias[o], 0.f));
        float h2[kHidden];
#pragma unroll
        for (int o = 0; o < kHidden; ++o) {
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < kHidden; ++c) a = fmaf(W2[o * kHidden + c], h1[c], a);
            h2[o] = bf16r(fmaxf(a + bias[kHidden + o], 0.f));
        }
        float out[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < kHidden; ++c) a = fmaf(W3[o * kHidden + c], h2[c], a);
            out[o] = a + bias[2 * kHidden + o];
        }
        int best = 0;
        float bv = out[0];
#pragma unroll
        for (int c = 1; c < kNumMat; ++c)
            if (out[c] > bv) { bv = out[c]; best = c; }
        const float wt = 1.0f / (1.0f + expf(-out[5]));
        const size_t o = (size_t)g * Q + q;
        mat[o] = (uint8_t)best;
        w[o] = wt;
        kappa[o] = mc.k[best];
        phi[o] = mc.phase[best];
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535 * 8) b = 65535 * 8;
    return (int)b;
}

}  // namespace

cudaError_t launch_decode_materials(const uint8_t* mats, int64_t n, MatConst mc, uint8_t* mat,
                                    float* w, float* kappa, float* phi, int* bad, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_decode_materials<<<grid_for(n, 256), 256, 0, s>>>(mats, n, mc, mat, w, kappa, phi, bad);
    return cudaGetLastError();
}

cudaError_t launch_decode_logits(const float* logits, int64_t n, MatConst mc, uint8_t* mat,
                                 float* w, float* kappa, float* phi, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_decode_logits<<<grid_for(n, 256), 256, 0, s>>>(logits, n, mc, mat, w, kappa, phi);
    return cudaGetLastError();
}

cudaError_t launch_decode_params(const uint8_t* mats, const float* w_in, const float* k_in,
                                 const float* p_in, int64_t n, uint8_t* mat, float* w,
                                 float* kappa, float* phi, int* bad, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_decode_params<<<grid_for(n, 256), 256, 0, s>>>(mats, w_in, k_in, p_in, n, mat, w, kappa,
                                                     phi, bad);
    return cudaGetLastError();
}

cudaError_t launch_decode_param_rows(const uint8_t* mats, const float* rows, int64_t V, int64_t n,
                                     uint8_t* mat, float* w, float* kappa, float* phi, int* bad,
                                     cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_decode_param_rows<<<grid_for(n, 256), 256, 0, s>>>(mats, rows, V, n, mat, w, kappa, phi, bad);
    return cudaGetLastError();
}

cudaError_t launch_pe_table(int nx, int ny, int nz, const float* B, void* pe_bf16, cudaStream_t s)
{
    const int n = nx * ny * nz * kPeRows;
    k_pe_table<<<(n + 255) / 256, 256, 0, s>>>(nx, ny, nz, B, (__nv_bfloat16*)pe_bf16);
    return cudaGetLastError();
}

cudaError_t launch_mlp_query_simt(int P, int Q, const void* pe_bf16, const float* genomes,
                                  MatConst mc, uint8_t* mat, float* w, float* kappa, float* phi,
                                  cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (kHidden * kPeDim + kHidden * kHidden + kOut * kHidden +
                                         2 * kHidden + kOut);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_simt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_simt<<<P, kSimtThreads, smem, s>>>(Q, (const __nv_bfloat16*)pe_bf16, genomes, mc, mat, w,
                                             kappa, phi);
    return cudaGetLastError();
}

}  // namespace vx
