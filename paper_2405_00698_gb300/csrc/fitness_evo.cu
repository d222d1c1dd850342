// Fitness reduction and the evolutionary step, fully on the GPU (Section II-C: "crossover,
// mutation and elite selection ... fully parallel"; Table I).
#include <cmath>

#include "common.cuh"

namespace vx {
namespace {

// ----------------------------------------------------------------------------------------------
// Fitness: centroid x displacement, FP64 warp-shuffle block reduction, one block per robot.
// The state is the displacement u from the rest pose, so the centroid displacement is the mean
// of u_x (u = 0 at the start).
// ----------------------------------------------------------------------------------------------
constexpr int kFitThreads = 256;

__global__ void __launch_bounds__(kFitThreads)
k_fitness(PopView pv, const int* __restrict__ mass_corner, const float4* __restrict__ u,
          const float4* __restrict__ x0, float dead_bound, double* __restrict__ out)
{
    __shared__ double sh_sum[kFitThreads / 32];
    __shared__ int sh_dead;
    const int r = blockIdx.x;
    const int M = pv.n_mass[r];
    const int64_t mo = pv.moff[r];
    if (threadIdx.x == 0) sh_dead = 0;
    __syncthreads();
    double s = 0.0;
    int dead = 0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int64_t c = mo + mass_corner[mo + m];
        const float4 d = u[c], r0 = x0[c];
        const float px = r0.x + d.x, py = r0.y + d.y, pz = r0.z + d.z;
        if (!(fabsf(px) <= dead_bound) || !(fabsf(py) <= dead_bound) || !(fabsf(pz) <= dead_bound))
            dead = 1;   // catches NaN too
        s += (double)d.x;
    }
    if (dead) sh_dead = 1;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh_sum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kFitThreads / 32; ++i) t += sh_sum[i];
        double f;
        if (M == 0) f = 0.0;
        else if (sh_dead) f = -INFINITY;
        else f = t / M;
        out[r] = f;
    }
}

// ----------------------------------------------------------------------------------------------
// Counter-based random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014).  Output
// number `ctr` of the stream seeded with `seed` is the SplitMix64 finaliser applied to
// seed + (ctr + 1) * golden-gamma.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr)
{
    uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

enum { kParentA = 0, kParentB = 1, kMask = 2, kMutate = 3, kU1 = 4, kU2 = 5, kCross = 6 };

// High 32 bits of the draw for (generation, child, gene, purpose), fields packed as
// generation | child (16 bits) | gene (26 bits) | purpose (3 bits).
__device__ __forceinline__ uint32_t draw32(uint64_t seed, uint64_t gen, uint32_t child,
                                           uint32_t gene, uint32_t purpose)
{
    const uint64_t ctr = ((((gen << 16) | child) << 26 | gene) << 3) | purpose;
    return (uint32_t)(splitmix64_at(seed, ctr) >> 32);
}

// Rank by counting: the rank of robot i is the number of robots ordered before it
// (larger fitness, or equal fitness and smaller index; NaN counts as -infinity).  The fitness
// values are compared as order-preserving 64-bit integer keys (the same order and the same ties
// as the floating-point comparison; -0 and +0 share a key), which runs on the integer pipes
// instead of the few FP64 units.
__device__ __forceinline__ unsigned long long rank_key(double x)
{
    if (isnan(x)) x = -INFINITY;
    if (x == 0.0) x = 0.0;                               // -0 and +0 compare equal
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_rank(const double* __restrict__ f, int P, int* __restrict__ order)
{
    extern __shared__ unsigned long long tile[];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long ki = i < P ? rank_key(f[i]) : 0ull;
    int rank = 0;
    for (int base = 0; base < P; base += blockDim.x) {
        __syncthreads();
        const int j = base + threadIdx.x;
        tile[threadIdx.x] = j < P ? rank_key(f[j]) : 0ull;
        __syncthreads();
        const int n = min((int)blockDim.x, P - base);
        if (i < P)
            for (int t = 0; t < n; ++t) {
                const unsigned long long kg = tile[t];
                const int jj = base + t;
                rank += (kg > ki) || (kg == ki && jj < i);
            }
    }
    if (i < P) order[rank] = i;
}

// One thread per (child row, gene).  Elite rows copy their genome; child rows pick parents,
// crossover mask and mutation from the counter-based generator.
__global__ void k_children(const float* __restrict__ gin, float* __restrict__ gout,
                           const int* __restrict__ order, int P, int G, int E, uint64_t seed,
                           uint64_t gen, uint32_t thresh, float sigma, uint32_t keep,
                           int* __restrict__ parents, uint8_t* __restrict__ mask)
{
    const int c = blockIdx.y;
    const size_t row = (size_t)c * G;
    if (c < E) {
        const float* src = gin + (size_t)order[c] * G;
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G; j += gridDim.x * blockDim.x) {
            gout[row + j] = src[j];
            if (mask) mask[row + j] = 0;
        }
        if (parents && blockIdx.x == 0 && threadIdx.x == 0) {
            parents[2 * c] = order[c];
            parents[2 * c + 1] = order[c];
        }
        return;
    }
    const uint32_t ua = draw32(seed, gen, c, 0, kParentA);
    const uint32_t ub = draw32(seed, gen, c, 0, kParentB);
    const int pa = order[(int)(((uint64_t)ua * (uint64_t)E) >> 32)];
    const int pb = order[(int)(((uint64_t)ub * (uint64_t)E) >> 32)];
    if (parents && blockIdx.x == 0 && threadIdx.x == 0) {
        parents[2 * c] = pa;
        parents[2 * c + 1] = pb;
    }
    const float* A = gin + (size_t)pa * G;
    const float* Bp = gin + (size_t)pb * G;
    // crossover rate below 1: some children copy parent A (a draw per child)
    const bool copy_a = keep != 0u && draw32(seed, gen, c, 0, kCross) < keep;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G; j += gridDim.x * blockDim.x) {
        const uint32_t m = copy_a ? 1u : draw32(seed, gen, c, j, kMask) >> 31;
        float g = m ? A[j] : Bp[j];
        if (draw32(seed, gen, c, j, kMutate) < thresh) {
            const float u1 = ((float)draw32(seed, gen, c, j, kU1) + 1.0f) * 2.3283064365386963e-10f;
            const float u2 = (float)draw32(seed, gen, c, j, kU2) * 2.3283064365386963e-10f;
            const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
            g = g + sigma * z;
        }
        gout[row + j] = g;
        if (mask) mask[row + j] = (uint8_t)m;
    }
}

// sin and cos of w t for the steps of one call, FP64 then rounded to float:
// phase = (2 pi freq) (step dt), evaluated in that order.
__global__ void k_sincos(double omega, double dt, int64_t step0, int n, float2* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = __dmul_rn((double)(step0 + i), dt);
    const double ph = __dmul_rn(omega, t);
    double s, c;
    sincos(ph, &s, &c);
    out[i] = make_float2((float)s, (float)c);
}

// Gather a per-mass float4 state into packed float[3] rows; `add` (optional) is added first
// (rest lattice + displacement = position).
__global__ void k_compact(PopView pv, const int* __restrict__ mass_corner,
                          const float4* __restrict__ src, const float4* __restrict__ add,
                          float* __restrict__ dst, const int64_t* __restrict__ dst_off)
{
    const int r = blockIdx.x;
    const int M = pv.n_mass[r];
    const int64_t mo = pv.moff[r], d = dst_off[r];
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int64_t c = mo + mass_corner[mo + m];
        float4 p = src[c];
        if (add) {
            const float4 q = add[c];
            p.x += q.x; p.y += q.y; p.z += q.z;
        }
        dst[3 * (d + m) + 0] = p.x;
        dst[3 * (d + m) + 1] = p.y;
        dst[3 * (d + m) + 2] = p.z;
    }
}

}  // namespace

cudaError_t launch_fitness(PopView pv, const int* mass_corner, const float4* u, const float4* x0,
                           float dead_bound, double* out, cudaStream_t s)
{
    if (pv.P == 0) return cudaSuccess;
    k_fitness<<<pv.P, kFitThreads, 0, s>>>(pv, mass_corner, u, x0, dead_bound, out);
    return cudaGetLastError();
}

namespace {

// dL/df weights of the E best robots in rank order (1 for the j-th ranked robot when j < E and
// its fitness is finite, 0 for every other robot).
__global__ void k_elite_weights(const int* __restrict__ order, const double* __restrict__ f, int P, int E,
                                double* __restrict__ w)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const int r = order[j];
    w[r] = (j < E && isfinite(f[r])) ? 1.0 : 0.0;
}

}  // namespace

cudaError_t launch_elite_weights(const int* order, const double* fitness, int P, int E, double* w, cudaStream_t s)
{
    k_elite_weights<<<(P + 255) / 256, 256, 0, s>>>(order, fitness, P, E, w);
    return cudaGetLastError();
}

cudaError_t launch_evo_rank(const double* fitness, int P, int* order, cudaStream_t s)
{
    const int T = 256;
    k_rank<<<(P + T - 1) / T, T, T * sizeof(unsigned long long), s>>>(fitness, P, order);
    return cudaGetLastError();
}

cudaError_t launch_evo_children(const float* gin, float* gout, const int* order, int P, int G,
                                int E, uint64_t seed, uint64_t gen, uint32_t thresh, float sigma,
                                uint32_t keep, int* parents, uint8_t* mask, cudaStream_t s)
{
    const int T = 256;
    int bx = (G + T - 1) / T;
    if (bx > 64) bx = 64;
    dim3 grid(bx, P);
    k_children<<<grid, T, 0, s>>>(gin, gout, order, P, G, E, seed, gen, thresh, sigma, keep, parents,
                                  mask);
    return cudaGetLastError();
}

cudaError_t launch_sincos_table(double omega, double dt, int64_t step0, int n, float2* out,
                                cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_sincos<<<(n + 255) / 256, 256, 0, s>>>(omega, dt, step0, n, out);
    return cudaGetLastError();
}

cudaError_t launch_compact_state(PopView pv, const int* mass_corner, const float4* src,
                                 const float4* add, float* dst, const int64_t* dst_off, cudaStream_t s)
{
    if (pv.P == 0) return cudaSuccess;
    k_compact<<<pv.P, 256, 0, s>>>(pv, mass_corner, src, add, dst, dst_off);
    return cudaGetLastError();
}

}  // namespace vx

// ----------------------------------------------------------------------------------------------
// Population diversity (logged per generation beside the fitness, Fig. 3(b) "diversity"):
//   genome: root of the mean pairwise squared distance, from the identity
//           mean_{i != j} |g_i - g_j|^2 = 2 P / (P - 1) * mean_i |g_i - mean g|^2;
//   morphology: mean over robot pairs of the fraction of voxels whose kept materials differ,
//           from per-voxel material counts c_k: differing pairs = (P^2 - sum_k c_k^2) / 2.
// FP64 accumulation; one block per gene / voxel chunk, atomics into two FP64 totals.
// ----------------------------------------------------------------------------------------------
namespace vx {
namespace {

__global__ void k_genome_spread(const float* __restrict__ g, int P, int G, double* __restrict__ total)
{
    double acc = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G; j += gridDim.x * blockDim.x) {
        double s = 0.0, s2 = 0.0;
        for (int i = 0; i < P; ++i) {
            const double x = (double)g[(size_t)i * G + j];
            s += x;
            s2 += x * x;
        }
        acc += s2 - s * s / P;             // sum_i (g_ij - mean_j)^2
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(total, acc);
}

__global__ void k_morph_spread(const uint8_t* __restrict__ mat, int P, int V, double* __restrict__ total)
{
    double acc = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        int c[kNumMat] = {0, 0, 0, 0, 0};
        for (int i = 0; i < P; ++i) c[mat[(size_t)i * V + v] % kNumMat]++;
        double eq = 0.0;
        for (int k = 0; k < kNumMat; ++k) eq += (double)c[k] * c[k];
        acc += ((double)P * P - eq) * 0.5;  // pairs of robots that differ at voxel v
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(total, acc);
}

}  // namespace

cudaError_t launch_diversity(const float* genomes, int P, int G, const uint8_t* mat, int V, double* totals,
                             cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(totals, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (genomes && G > 0) k_genome_spread<<<std::min((G + 255) / 256, 1024), 256, 0, s>>>(genomes, P, G, totals);
    if (mat && V > 0) k_morph_spread<<<std::min((V + 255) / 256, 1024), 256, 0, s>>>(mat, P, V, totals + 1);
    return cudaGetLastError();
}

}  // namespace vx

// ----------------------------------------------------------------------------------------------
// Lamarckian gradient step on genome rows [w | kappa | phi] (gradient-assisted co-design): for
// listed row r and gene j, genome <- clamp(fmaf(eta_seg, d, genome), lo_j, hi_j) with d the
// adjoint's gradient of voxel j mod V of robot r (robot r's voxels start at voff[r]) and eta_seg
// the step of the gene's segment.
// ----------------------------------------------------------------------------------------------
namespace vx {
namespace {

__global__ void k_grad_step(float* __restrict__ genomes, int G, int64_t V, const int64_t* __restrict__ voff,
                            const float* __restrict__ g_w, const float* __restrict__ g_kappa,
                            const float* __restrict__ g_phi, const int* __restrict__ rows, float eta_w,
                            float eta_kappa, float eta_phi, const float* __restrict__ lo,
                            const float* __restrict__ hi)
{
    const int r = rows[blockIdx.y];
    float* row = genomes + (size_t)r * G;
    const int64_t base = voff[r];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G; j += gridDim.x * blockDim.x) {
        const int seg = (int)(j / V);
        const int64_t v = j - seg * V;
        const float* grad = seg == 0 ? g_w : (seg == 1 ? g_kappa : g_phi);
        const float eta = seg == 0 ? eta_w : (seg == 1 ? eta_kappa : eta_phi);
        float x = __fmaf_rn(eta, grad[base + v], row[j]);
        if (lo) x = fmaxf(x, lo[j]);
        if (hi) x = fminf(x, hi[j]);
        row[j] = x;
    }
}

}  // namespace

cudaError_t launch_grad_step(float* genomes, int G, int64_t V, const int64_t* voff, const float* g_w,
                             const float* g_kappa, const float* g_phi, const int* rows, int n_rows,
                             float eta_w, float eta_kappa, float eta_phi, const float* lo,
                             const float* hi, cudaStream_t s)
{
    if (n_rows == 0 || G == 0) return cudaSuccess;
    const int T = 256;
    int bx = (G + T - 1) / T;
    if (bx > 64) bx = 64;
    k_grad_step<<<dim3(bx, n_rows), T, 0, s>>>(genomes, G, V, voff, g_w, g_kappa, g_phi, rows, eta_w,
                                               eta_kappa, eta_phi, lo, hi);
    return cudaGetLastError();
}

}  // namespace vx
