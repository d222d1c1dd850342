// MLP spatial query on the 5th-generation tensor cores (Section II-C: "the material score from
// the model's Softmax branch will determine the material category and the material weight from
// the model's Sigmoid branch will be multiplied by the material parameters"; Eq. (1) gives the
// input encoding).
//
// Per genome: gamma [Q x 256] -> ReLU(. W1^T + b1) [Q x 64] -> ReLU(. W2^T + b2) [Q x 64]
// -> (. W3^T + b3) [Q x 6]; material = argmax of outputs 0..4 (softmax is monotone; ties to the
// lowest id), weight = sigmoid(output 5).
//
// One CTA (4 warps) per genome at a time, persistent over genomes, two CTAs per SM (one CTA's
// weight conversion and epilogues overlap the other's tensor work; measured 1.6x over one CTA
// per SM with a double-buffered gamma tile).  Shared-memory operands are bfloat16 in the
// 128-byte-swizzled K-major layout the tensor core reads directly (107 KB per CTA):
//   * gamma tiles of 128 queries arrive by TMA into one buffer; the next tile's copy is issued
//     as soon as layer 1 has read the current one, so it overlaps the rest of the tile;
//   * W1, W2, W3 are converted from the float32 genome by the CTA's threads into that layout
//     (W3 padded to 16 rows);
//   * the three layers are tcgen05.mma kind::f16 (M = 128; N = 64, 64, 16) accumulating in
//     TMEM; one thread issues them; completion is signalled on an mbarrier by tcgen05.commit;
//   * each epilogue reads its accumulator rows with tcgen05.ld (warp w owns TMEM lanes
//     32w..32w+31 = queries of the tile), adds the bias, applies ReLU, rounds to bfloat16 and
//     stores the hidden activations in TMEM with tcgen05.st (row i in lane i, two units per
//     column), where layers 2 and 3 read their A operand; the last epilogue computes the heads
//     and writes material, weight, stiffness and phase per voxel.
// Every mbarrier wait is bounded: on timeout the kernel raises a status bit, abandons the
// remaining work and still releases its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace vx {
namespace {

constexpr int kThreads = 128;
constexpr int kTileM = 128;
constexpr int kKBlock = 64;                                  // bf16 per 128-byte swizzle row
constexpr int kABytes = kTileM * kPeDim * 2;                 // 64 KB: one gamma tile
constexpr int kW1Bytes = kHidden * kPeDim * 2;               // 32 KB
constexpr int kW2Bytes = kHidden * kHidden * 2;              // 8 KB
constexpr int kW3Rows = 16;
constexpr int kW3Bytes = kW3Rows * kHidden * 2;              // 2 KB
constexpr int kTmemCols = 256;
constexpr uint32_t kSpinLimit = 1u << 24;

struct __align__(1024) Smem {
    unsigned char a[1][kABytes];          // gamma tile; after layer 1 also the hidden activations
    unsigned char w1[kW1Bytes];
    unsigned char w2[kW2Bytes];
    unsigned char w3[kW3Bytes];
    float b1[kHidden];
    float b2[kHidden];
    float b3[kW3Rows];
    uint64_t tma_bar[2];
    uint64_t mma_bar;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of a K-major bfloat16 operand stored as 64-wide K blocks of
// `rows` x 128 bytes, with the 128-byte swizzle (16-byte chunk j of row r at chunk j ^ (r % 8)).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k, int rows)
{
    const int kb = k / kKBlock, kk = k % kKBlock;
    const int chunk = (kk >> 3) ^ (row & 7);
    return (uint32_t)(kb * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 + chunk * 16 + (kk & 7) * 2);
}

// Shared-memory matrix descriptor of a 128-byte-swizzled K-major operand starting at `addr`
// (rows grouped by 8 at a 1024-byte stride).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);     // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16, bfloat16 A and B (K-major), float32 accumulator, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; gives up (and flags the CTA) after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, Smem& s, int* status)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, phase)) return true;
        if (*(volatile int*)&s.abort) return false;
    }
    *(volatile int*)&s.abort = 1;
    atomicOr(status, 4);
    return false;
}

// Bounded wait on an mbarrier phase that ignores the abort flag: after an abort, the issuing
// thread waits (again at most kSpinLimit polls) for the copy or MMA it still has in flight before
// the CTA frees its tensor memory and exits.  Returns whether the phase completed.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t phase)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                     uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

// The same with the A operand (M x 16 bfloat16, row i in lane i, two elements per column) read
// from tensor memory at column address a_tmem.
__device__ __forceinline__ void umma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit columns of TMEM into 16 registers of each thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive 32-bit columns of this thread's lane from 32 registers, then wait for them.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
          "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
          "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&p);
}

// Convert a float32 [rows][K] weight block (8-byte aligned) into the swizzled bf16 layout.
// Each thread takes kUnroll chunks of 8 values per round and issues all their loads before
// converting any, so several global loads per thread are in flight.
constexpr int kUnroll = 8;
__device__ __forceinline__ void load_weights(const float* __restrict__ src, int rows, int K,
                                             int valid_rows, unsigned char* dst)
{
    const int chunks = rows * (K / 8);
    for (int c0 = threadIdx.x; c0 < chunks; c0 += kThreads * kUnroll) {
        float2 v[kUnroll][4];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int c = c0 + u * kThreads;
            const int row = c / (K / 8), k0 = (c % (K / 8)) * 8;
            if (c < chunks && row < valid_rows) {
                const float2* p = reinterpret_cast<const float2*>(src + (size_t)row * K + k0);
                v[u][0] = p[0]; v[u][1] = p[1]; v[u][2] = p[2]; v[u][3] = p[3];
            } else {
                v[u][0] = v[u][1] = v[u][2] = v[u][3] = make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int c = c0 + u * kThreads;
            const int row = c / (K / 8), k0 = (c % (K / 8)) * 8;
            if (c < chunks)
                *reinterpret_cast<uint4*>(dst + sw128_offset(row, k0, rows)) =
                    make_uint4(pack_bf16(v[u][0].x, v[u][0].y), pack_bf16(v[u][1].x, v[u][1].y),
                               pack_bf16(v[u][2].x, v[u][2].y), pack_bf16(v[u][3].x, v[u][3].y));
        }
    }
}

// Bias + ReLU of a 64-wide accumulator row block, rounded to bfloat16 and stored as the next
// layer's A operand in tensor memory (this thread's lane = query row of the tile; column j holds
// hidden units 2j and 2j + 1, the lower index in the low half).
__device__ __forceinline__ void epilogue_hidden(uint32_t taddr, const float* bias, uint32_t th)
{
    uint32_t p[32];
#pragma unroll
    for (int c0 = 0; c0 < kHidden; c0 += 16) {
        float v[16];
        tmem_ld16(taddr + c0, v);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            p[c0 / 2 + i] = pack_bf16(fmaxf(v[2 * i] + bias[c0 + 2 * i], 0.f),
                                      fmaxf(v[2 * i + 1] + bias[c0 + 2 * i + 1], 0.f));
    }
    tmem_st32(th, p);
}

__global__ void __launch_bounds__(kThreads, 2)
k_mlp_tc(const __grid_constant__ CUtensorMap pe_map, int P, int Q, const float* __restrict__ genomes,
         MatConst mc, uint8_t* __restrict__ mat, float* __restrict__ w_out, float* __restrict__ kappa,
         float* __restrict__ phi, int* status)
{
    extern __shared__ unsigned char smem_raw[];
    Smem& s = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s.tmem_base)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&s.tma_bar[0], 1);
        mbar_init(&s.tma_bar[1], 1);
        mbar_init(&s.mma_bar, 1);
        s.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    // accumulators of the three layers, then the hidden activations (bf16 pairs), which are the
    // A operand of layers 2 and 3
    const uint32_t t_d1 = tmem, t_d2 = tmem + 64, t_d3 = tmem + 128, t_h = tmem + 160;
    const uint32_t lane_sel = (uint32_t)(warp * 32) << 16;    // this warp's TMEM lane quarter
    const int ntiles = (Q + kTileM - 1) / kTileM;
    uint32_t tma_phase = 0, mma_phase = 0;
    constexpr uint32_t id_h = idesc_bf16(kTileM, kHidden);
    constexpr uint32_t id_o = idesc_bf16(kTileM, kW3Rows);
    // issuing thread only: the TMA batch and the MMA commit whose completion it has not yet
    // observed (at most one of each: nothing new is issued once the CTA has aborted)
    bool tma_out = false, mma_out = false;
    uint32_t tma_out_phase = 0, mma_out_phase = 0;
    bool stop = false;
    // the gamma tile of the next layer-1 MMA, copied as soon as the buffer is free (right after
    // the previous tile's layer 1), so the copy overlaps that tile's epilogues and layers 2, 3
    auto issue_gamma = [&](int tile) {
        mbar_expect_tx(&s.tma_bar[0], kABytes);
        for (int kb = 0; kb < kPeDim / kKBlock; ++kb)
            tma_load_2d(s.a[0] + kb * kTileM * 128, &pe_map, &s.tma_bar[0], kb * kKBlock, tile * kTileM);
        tma_out = true;
        tma_out_phase = tma_phase;
    };
    if (tid == 0 && (int)blockIdx.x < P) issue_gamma(0);

    for (int g = blockIdx.x; g < P && !stop; g += gridDim.x) {
        const float* G = genomes + (size_t)g * kGenome;
        load_weights(G + kOffW1, kHidden, kPeDim, kHidden, s.w1);
        load_weights(G + kOffW2, kHidden, kHidden, kHidden, s.w2);
        load_weights(G + kOffW3, kW3Rows, kHidden, kOut, s.w3);
        for (int i = tid; i < kHidden; i += kThreads) {
            s.b1[i] = G[kOffB1 + i];
            s.b2[i] = G[kOffB2 + i];
        }
        if (tid < kW3Rows) s.b3[tid] = tid < kOut ? G[kOffB3 + tid] : 0.f;
        proxy_fence();
        __syncthreads();
        for (int t = 0; t < ntiles; ++t) {
            // layer 1: D1 = gamma_tile . W1^T  (K = 256: 4 swizzle blocks x 4 steps of 16)
            if (tid == 0 && tma_out && !s.abort) {
                if (mbar_wait(&s.tma_bar[0], tma_phase, s, status)) {
                    tma_out = false;
                    tma_phase ^= 1;
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(s.a[0]), b0 = smem_u32(s.w1);
#pragma unroll
                    for (int k = 0; k < kPeDim / 16; ++k) {
                        const uint32_t ao = (k / 4) * (kTileM * 128) + (k % 4) * 32;
                        const uint32_t bo = (k / 4) * (kHidden * 128) + (k % 4) * 32;
                        umma(t_d1, sw128_desc(a0 + ao), sw128_desc(b0 + bo), id_h, k > 0);
                    }
                    umma_commit(&s.mma_bar);
                    mma_out = true;
                    mma_out_phase = mma_phase;
                }
            }
            const int row = warp * 32 + lane;
            if (mbar_wait(&s.mma_bar, mma_phase, s, status) && tid == 0) mma_out = false;
            mma_phase ^= 1;
            // the gamma buffer is free again: the next tile's copy (or the next genome's first)
            if (tid == 0 && !s.abort && (t + 1 < ntiles || g + (int)gridDim.x < P))
                issue_gamma(t + 1 < ntiles ? t + 1 : 0);
            // epilogue 1 -> H (tensor memory)
            tc_fence_after();
            if (!s.abort) epilogue_hidden(t_d1 + lane_sel, s.b1, t_h + lane_sel);
            tc_fence_before();
            __syncthreads();
            // layer 2: D2 = H . W2^T, H read from tensor memory (8 columns per step of K = 16)
            if (tid == 0 && !s.abort) {
                tc_fence_after();
                const uint32_t b0 = smem_u32(s.w2);
#pragma unroll
                for (int k = 0; k < kHidden / 16; ++k)
                    umma_ts(t_d2, t_h + k * 8, sw128_desc(b0 + k * 32), id_h, k > 0);
                umma_commit(&s.mma_bar);
                mma_out = true;
                mma_out_phase = mma_phase;
            }
            if (mbar_wait(&s.mma_bar, mma_phase, s, status) && tid == 0) mma_out = false;
            mma_phase ^= 1;
            tc_fence_after();
            if (!s.abort) epilogue_hidden(t_d2 + lane_sel, s.b2, t_h + lane_sel);
            tc_fence_before();
            __syncthreads();
            // layer 3: D3 = H . W3^T (N = 16, rows 6..15 of W3 are zero)
            if (tid == 0 && !s.abort) {
                tc_fence_after();
                const uint32_t b0 = smem_u32(s.w3);
#pragma unroll
                for (int k = 0; k < kHidden / 16; ++k)
                    umma_ts(t_d3, t_h + k * 8, sw128_desc(b0 + k * 32), id_o, k > 0);
                umma_commit(&s.mma_bar);
                mma_out = true;
                mma_out_phase = mma_phase;
            }
            if (mbar_wait(&s.mma_bar, mma_phase, s, status) && tid == 0) mma_out = false;
            mma_phase ^= 1;
            tc_fence_after();
            if (!s.abort) {
                float o[16];
                tmem_ld16(t_d3 + lane_sel, o);
                const int q = t * kTileM + row;
                if (q < Q) {
                    int best = 0;
                    float bv = o[0] + s.b3[0];
#pragma unroll
                    for (int c = 1; c < kNumMat; ++c) {
                        const float x = o[c] + s.b3[c];
                        if (x > bv) { bv = x; best = c; }
                    }
                    const float wt = 1.0f / (1.0f + expf(-(o[5] + s.b3[5])));
                    const size_t idx = (size_t)g * Q + q;
                    mat[idx] = (uint8_t)best;
                    w_out[idx] = wt;
                    kappa[idx] = mc.k[best];
                    phi[idx] = mc.phase[best];
                }
            }
            tc_fence_before();
            // one decision for the whole CTA: after an abort no thread touches the tiles again
            if (__syncthreads_or(s.abort)) { stop = true; break; }
        }
    }
    // after an abort the issuing thread first waits (bounded) for its copy and MMA still in
    // flight, so the tensor memory is not freed under an MMA and no copy lands in the shared
    // memory of an exited CTA
    if (tid == 0 && stop) {
        if (tma_out) mbar_drain(&s.tma_bar[0], tma_out_phase);
        if (mma_out) mbar_drain(&s.mma_bar, mma_out_phase);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

}  // namespace

size_t mlp_tc_smem_bytes() { return sizeof(Smem) + 1024; }

cudaError_t launch_mlp_query(int P, int Q, const void* pe_bf16, const float* genomes, MatConst mc,
                             uint8_t* mat, float* w, float* kappa, float* phi, int* status,
                             int num_sms, cudaStream_t s)
{
    if (P == 0 || Q == 0) return cudaSuccess;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // gamma table [Q][256] bfloat16, row stride 512 B; boxes of 64 x 128, 128-byte swizzle
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)kPeDim, (cuuint64_t)Q};
    const cuuint64_t strides[1] = {(cuuint64_t)kPeDim * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKBlock, (cuuint32_t)kTileM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(pe_bf16), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const size_t smem = mlp_tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = P < 2 * num_sms ? P : 2 * num_sms;
    k_mlp_tc<<<grid, kThreads, smem, s>>>(map, P, Q, genomes, mc, mat, w, kappa, phi, status);
    return cudaGetLastError();
}

}  // namespace vx
