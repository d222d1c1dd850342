// Reverse-mode adjoint for streamed robots (too large to keep on one SM): the same gradient as
// the resident lattice adjoint (d sum_r dL_df[r] fitness_r / d per-voxel w, kappa, phi), with
// the state kept in device memory.  The forward run checkpoints the state every K steps; the
// backward replays each segment with the streamed step kernel in recording mode (state before
// the update, contact mode, horizontal force before contact), then sweeps it backwards one
// launch per step.  A launch does, for every mass corner:
//   spring part of step j: from its own and its neighbours' recorded positions and adjoint
//     forces, each forward spring's transpose (lambda_u -= ..., sensitivity sums += ...) and each
//     backward spring's (lambda_u += ...), in direction order as the resident adjoint;
//   mass part of step j - 1: the transpose of that step's mass update, which needs only the
//     corner's own adjoints, giving the adjoint force the next launch reads from its neighbours
//     (two buffers, so no launch reads what it writes).
// Every spring's sensitivity sums belong to its lower corner, so no atomics are needed until the
// final scatter onto voxels.
#include "adjoint.cuh"
#include "common.cuh"
#include "physics.cuh"

namespace vx {
namespace {

constexpr int kAdjThreads = 256;

struct CornerRef {
    int r, X, XY, C, cidx;
    int64_t mo;
    uint32_t fl;
};

// NC > 0: every streamed robot is NC x NC x NC (compile-time strides, as in the forward step).
template <int NC = 0>
__device__ __forceinline__ bool corner_ref(const StreamAdjArgs& a, CornerRef& q)
{
    q.r = a.robots[blockIdx.y];
    const int nx = a.pv.dims[3 * q.r], ny = a.pv.dims[3 * q.r + 1], nz = a.pv.dims[3 * q.r + 2];
    q.X = NC ? NC + 1 : nx + 1;
    q.XY = NC ? (NC + 1) * (NC + 1) : (nx + 1) * (ny + 1);
    q.C = NC ? (NC + 1) * (NC + 1) * (NC + 1) : q.XY * (nz + 1);
    q.cidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (q.cidx >= q.C) return false;
    q.mo = a.pv.moff[q.r];
    q.fl = a.cflags[q.mo + q.cidx];
    return (q.fl >> 31) != 0u;                  // corners without a mass take no part
}

// Adjoint of the final state (the fitness is the mean of u_x over the masses) and zero sums.
__global__ void __launch_bounds__(kAdjThreads) k_sadj_init(StreamAdjArgs a)
{
    CornerRef q;
    if (!corner_ref(a, q)) return;
    const int M = a.pv.n_mass[q.r];
    const int64_t o = q.mo + q.cidx;
    a.lu[o] = make_float4((float)(a.dL_df[q.r] / (double)M), 0.f, 0.f, 0.f);
    a.lv[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    float* acc = a.acc + 39 * q.mo;
    for (int k = 0; k < 39; ++k) acc[k * q.C + q.cidx] = 0.f;
}

template <int NC>
__global__ void __launch_bounds__(kAdjThreads, 4) k_sadj_step(StreamAdjArgs a)
{
    CornerRef q;
    if (!corner_ref<NC>(a, q)) return;
    const int64_t o = q.mo + q.cidx;
    const int X = q.X, XY = q.XY, C = q.C, cidx = q.cidx;
    const uint32_t fl = q.fl;
    const StepConst c = a.c;
    float4 lu = a.lu[o];
    float lux = lu.x, luy = lu.y, luz = lu.z;
    if (a.step >= 0) {
        // ---- spring part of step j ----
        const float4* __restrict__ ru = a.rec_u + q.mo;
        const float4* __restrict__ lFin = a.lF_in + q.mo;
        const float* __restrict__ prm = a.prm + 39 * q.mo;
        float* __restrict__ acc = a.acc + 39 * q.mo;
        const float4 un = ru[cidx];
        const float4 lF = lFin[cidx];
        const float2 sc = a.sc[a.step];
        // loads of 3 directions are issued before they are used; absent springs load nothing
        // (far end = the corner itself, k = 0: their transposes are exact zeros).  With at least
        // 4 blocks per SM, 25 % less time than loads behind each direction's mask test.
        for_each_batch<3>([&](auto t0) {       // own forward springs: a = c, b = c + offset
            constexpr int d0 = decltype(t0)::value;
            constexpr int nbt = d0 + 3 <= 13 ? 3 : 13 - d0;
            float4 ub[nbt], gb[nbt];
            float pk[nbt], pa[nbt], pb[nbt], sk[nbt], sa[nbt], sb[nbt];
            for_each_dir_in<d0, nbt>([&](auto t) {
                constexpr int d = decltype(t)::value, i = d - d0;
                const bool has = (fl >> d) & 1u;
                const int nb = cidx + lattice_offset<d>(X, XY);
                ub[i] = has ? ru[nb] : un;
                gb[i] = has ? lFin[nb] : lF;
                pk[i] = has ? prm[d * C + cidx] : 0.f;
                pa[i] = has ? prm[(13 + d) * C + cidx] : 0.f;
                pb[i] = has ? prm[(26 + d) * C + cidx] : 0.f;
                sk[i] = has ? acc[d * C + cidx] : 0.f;
                sa[i] = has ? acc[(13 + d) * C + cidx] : 0.f;
                sb[i] = has ? acc[(26 + d) * C + cidx] : 0.f;
            });
            for_each_dir_in<d0, nbt>([&](auto t) {
                constexpr int d = decltype(t)::value, i = d - d0;
                const SpringEval e = spring_eval_dir<d>(
                    __fsub_rn(ub[i].x, un.x), __fsub_rn(ub[i].y, un.y), __fsub_rn(ub[i].z, un.z), c.edge,
                    lattice_rest<d>(c), lattice_rest_sq<d>(c), pk[i], pa[i], pb[i], sc.x, sc.y);
                float ldx, ldy, ldz, dk, da, db;
                spring_adjoint(e, pk[i], lF.x - gb[i].x, lF.y - gb[i].y, lF.z - gb[i].z, sc.x, sc.y, ldx, ldy, ldz,
                               dk, da, db);
                lux -= ldx; luy -= ldy; luz -= ldz;
                if ((fl >> d) & 1u) {
                    acc[d * C + cidx] = sk[i] + dk;
                    acc[(13 + d) * C + cidx] = sa[i] + da;
                    acc[(26 + d) * C + cidx] = sb[i] + db;
                }
            });
        });
        for_each_batch<3>([&](auto t0) {       // backward springs: a = c - offset, b = c
            constexpr int d0 = decltype(t0)::value;
            constexpr int nbt = d0 + 3 <= 13 ? 3 : 13 - d0;
            float4 ua[nbt], ga[nbt];
            float pk[nbt], pa[nbt], pb[nbt];
            for_each_dir_in<d0, nbt>([&](auto t) {
                constexpr int d = decltype(t)::value, i = d - d0;
                const bool has = (fl >> (16 + d)) & 1u;
                const int na = cidx - lattice_offset<d>(X, XY);
                ua[i] = has ? ru[na] : un;
                ga[i] = has ? lFin[na] : lF;
                pk[i] = has ? prm[d * C + na] : 0.f;
                pa[i] = has ? prm[(13 + d) * C + na] : 0.f;
                pb[i] = has ? prm[(26 + d) * C + na] : 0.f;
            });
            for_each_dir_in<d0, nbt>([&](auto t) {
                constexpr int d = decltype(t)::value, i = d - d0;
                const SpringEval e = spring_eval_dir<d>(
                    __fsub_rn(un.x, ua[i].x), __fsub_rn(un.y, ua[i].y), __fsub_rn(un.z, ua[i].z), c.edge,
                    lattice_rest<d>(c), lattice_rest_sq<d>(c), pk[i], pa[i], pb[i], sc.x, sc.y);
                float ldx, ldy, ldz, dk, da, db;
                spring_adjoint(e, pk[i], ga[i].x - lF.x, ga[i].y - lF.y, ga[i].z - lF.z, sc.x, sc.y, ldx, ldy, ldz,
                               dk, da, db);
                lux += ldx; luy += ldy; luz += ldz;
            });
        });
    }
    if (a.mrec_u) {
        // ---- mass part of step j - 1 ----
        const float4 un = a.mrec_u[o];
        const float2 fh = a.mrec_f[o];
        const float4 lv = a.lv[o];
        float lvx = lv.x, lvy = lv.y, lvz = lv.z;
        float lFx = 0.f, lFy = 0.f, lFz = 0.f;
        mass_adjoint(__float_as_uint(un.w), a.u0[o].w + un.z, fh, lux, luy, luz, lvx, lvy, lvz, lFx, lFy, lFz, c);
        a.lv[o] = make_float4(lvx, lvy, lvz, 0.f);
        a.lF_out[o] = make_float4(lFx, lFy, lFz, 0.f);
    }
    a.lu[o] = make_float4(lux, luy, luz, 0.f);
}

// Per forward spring: its sensitivity sums onto the incident voxels.
__global__ void __launch_bounds__(kAdjThreads) k_sadj_voxels(StreamAdjArgs a)
{
    CornerRef q;
    if (!corner_ref(a, q)) return;
    const int nx = a.pv.dims[3 * q.r], ny = a.pv.dims[3 * q.r + 1], nz = a.pv.dims[3 * q.r + 2];
    const int64_t vo = a.pv.voff[q.r];
    const float* acc = a.acc + 39 * q.mo;
    for_each_dir([&](auto t) {
        constexpr int d = decltype(t)::value;
        if (!((q.fl >> d) & 1u)) return;
        spring_sens_to_voxels<d>(q.cidx, q.X, q.XY, nx, ny, nz, a.mat + vo, acc[d * q.C + q.cidx],
                                 acc[(13 + d) * q.C + q.cidx], acc[(26 + d) * q.C + q.cidx], a.c,
                                 a.g_k + vo, a.g_a + vo, a.g_b + vo);
    });
}

dim3 grid_of(const StreamAdjArgs& a, int max_corners)
{
    return dim3((max_corners + kAdjThreads - 1) / kAdjThreads, a.n_robots);
}

}  // namespace

cudaError_t launch_stream_adj_init(const StreamAdjArgs& a, int max_corners, cudaStream_t s)
{
    if (a.n_robots == 0) return cudaSuccess;
    k_sadj_init<<<grid_of(a, max_corners), kAdjThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stream_adj_step(const StreamAdjArgs& a, int max_corners, cudaStream_t s)
{
    if (a.n_robots == 0) return cudaSuccess;
    if (a.cube40) k_sadj_step<40><<<grid_of(a, max_corners), kAdjThreads, 0, s>>>(a);
    else k_sadj_step<0><<<grid_of(a, max_corners), kAdjThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stream_adj_voxels(const StreamAdjArgs& a, int max_corners, cudaStream_t s)
{
    if (a.n_robots == 0) return cudaSuccess;
    k_sadj_voxels<<<grid_of(a, max_corners), kAdjThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vx
