// Streamed time stepping for robots too large to keep on one SM (Section II-C: the spring and
// mass updates of one step; Table II constants).  State lives in device memory as per-corner
// float4 arrays (structure of arrays over the whole lattice of every robot); one launch advances
// every corner of every streamed robot by one step:
//   thread = one grid corner (consecutive threads = consecutive corners, coalesced);
//   it evaluates its forward springs (own parameters) and its backward springs (the lower
//   endpoint's parameters, read from the same coalesced planes at corner c - offset(d)), each
//   with the shared arithmetic of physics.cuh and in the same order as the lattice kernel, so a
//   robot stepped here follows the resident path's trajectory bit for bit;
//   positions and velocities are double-buffered (read *_in, write *_out), so one launch needs
//   no grid-wide barrier.
// Per spring update it moves the spring's parameters twice (once per endpoint, 24 B) and the
// endpoint states through L2; per corner 16 B in + 32 B out (u, v) + 16 B v in + 4 B flags.
#include "common.cuh"
#include "physics.cuh"

namespace vx {
namespace {

// Loads of 3 directions in flight per batch and at least 8 blocks of 128 threads per SM (64
// registers, no spills): measured 0.137 ms per step on 32 robots 40x40x40.  With 4 blocks of 256
// threads: 0.140 ms, against 0.159 ms for batches of 4, 0.155 / 0.140 / 0.154 / 0.266 ms for
// batches of 2 / 5 / 7 / 13, and 0.175 / 0.173 ms with 3 / 5 blocks per SM (batches of 3 / 5);
// 2 blocks of 512 threads 0.145 ms, 10 blocks of 128 (48 registers, spills) 0.163 ms.
constexpr int kStreamThreads = 128;
constexpr int kStreamBatch = 3;
constexpr int kStreamMinBlocks = 8;

// NC > 0: every robot of the launch is NC x NC x NC (the large-robot workload's 40^3 grid): the
// strides and plane size are compile-time constants, so the 13 neighbour and 39 parameter
// addresses are immediate offsets (12.7 % faster on 64 robots 40^3, same bits).
template <int NC>
__global__ void __launch_bounds__(kStreamThreads, kStreamMinBlocks)
k_step_streamed(StreamArgs a, int n)
{
    const int r = a.robots[blockIdx.y];
    const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
    const int X = NC ? NC + 1 : nx + 1, XY = NC ? (NC + 1) * (NC + 1) : (nx + 1) * (ny + 1),
              C = NC ? (NC + 1) * (NC + 1) * (NC + 1) : XY * (nz + 1);
    const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (cidx >= C) return;
    const int64_t mo = a.pv.moff[r];
    const uint32_t fl = a.cflags[mo + cidx];
    if (!(fl >> 31)) return;                    // no mass here: nothing moves
    const float4* __restrict__ uin = a.u_in + mo;
    float4 u = uin[cidx];
    const float4* __restrict__ vin = a.v_in + mo;
    float4 v = vin[cidx];
    if (a.ckpt_u) {                             // state at the start of a checkpointed segment
        a.ckpt_u[mo + cidx] = u;
        a.ckpt_v[mo + cidx] = v;
    }
    const float* __restrict__ prm = a.prm + 39 * mo;
    const float2 sc = a.sc[n];
    const StepConst c = a.c;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    // Loads are issued for a batch of directions before any of them is evaluated: the
    // memory-level parallelism the per-step pass needs.  An absent spring's loads are predicated
    // off (its far end is the corner's own u, its parameters zero: 5 % less time than loading
    // them) and its evaluation takes no branch (another 5 %): du = 0 and k = 0 make its force an
    // exact zero that leaves the sums' bits unchanged.  The sums keep the fixed order (forward by
    // direction, then backward by direction).
    // the 40^3 instantiation, with its addresses constant, has the registers for batches of five
    // directions (1.098x over three; six spill)
    constexpr int kBatch = NC ? 5 : kStreamBatch;
    for_each_batch<kBatch>([&](auto t0) {      // forward springs (c, c + offset(d))
        constexpr int d0 = decltype(t0)::value;
        constexpr int nb = d0 + kBatch <= 13 ? kBatch : 13 - d0;
        float4 ub[nb];
        float pk[nb], pa[nb], pb[nb];
        for_each_dir_in<d0, nb>([&](auto t) {
            constexpr int d = decltype(t)::value, i = d - d0;
            const bool has = (fl >> d) & 1u;
            ub[i] = has ? uin[cidx + lattice_offset<d>(X, XY)] : u;
            pk[i] = has ? prm[d * C + cidx] : 0.f;
            pa[i] = has ? prm[(13 + d) * C + cidx] : 0.f;
            pb[i] = has ? prm[(26 + d) * C + cidx] : 0.f;
        });
        for_each_dir_in<d0, nb>([&](auto t) {
            constexpr int d = decltype(t)::value, i = d - d0;
            SpringEval e = spring_eval_dir<d>(__fsub_rn(ub[i].x, u.x), __fsub_rn(ub[i].y, u.y), __fsub_rn(ub[i].z, u.z),
                                              c.edge, lattice_rest<d>(c), lattice_rest_sq<d>(c), pk[i], pa[i], pb[i], sc.x, sc.y);
            if (c.damped) {
                const float4 vb = vin[((fl >> d) & 1u) ? cidx + lattice_offset<d>(X, XY) : cidx];
                spring_dashpot(e, __fsub_rn(vb.x, v.x), __fsub_rn(vb.y, v.y), __fsub_rn(vb.z, v.z), pk[i], c);
            }
            Fx = __fadd_rn(Fx, e.gx); Fy = __fadd_rn(Fy, e.gy); Fz = __fadd_rn(Fz, e.gz);
        });
    });
    for_each_batch<kBatch>([&](auto t0) {      // backward springs (c - offset(d), c)
        constexpr int d0 = decltype(t0)::value;
        constexpr int nb = d0 + kBatch <= 13 ? kBatch : 13 - d0;
        float4 ua[nb];
        float pk[nb], pa[nb], pb[nb];
        for_each_dir_in<d0, nb>([&](auto t) {
            constexpr int d = decltype(t)::value, i = d - d0;
            const bool has = (fl >> (16 + d)) & 1u;
            const int na = has ? cidx - lattice_offset<d>(X, XY) : cidx;
            ua[i] = has ? uin[na] : u;
            pk[i] = has ? prm[d * C + na] : 0.f;
            pa[i] = has ? prm[(13 + d) * C + na] : 0.f;
            pb[i] = has ? prm[(26 + d) * C + na] : 0.f;
        });
        for_each_dir_in<d0, nb>([&](auto t) {
            constexpr int d = decltype(t)::value, i = d - d0;
            SpringEval e = spring_eval_dir<d>(__fsub_rn(u.x, ua[i].x), __fsub_rn(u.y, ua[i].y), __fsub_rn(u.z, ua[i].z),
                                              c.edge, lattice_rest<d>(c), lattice_rest_sq<d>(c), pk[i], pa[i], pb[i], sc.x, sc.y);
            if (c.damped) {
                const float4 va = vin[((fl >> (16 + d)) & 1u) ? cidx - lattice_offset<d>(X, XY) : cidx];
                spring_dashpot(e, __fsub_rn(v.x, va.x), __fsub_rn(v.y, va.y), __fsub_rn(v.z, va.z), pk[i], c);
            }
            Fx = __fadd_rn(Fx, -e.gx); Fy = __fadd_rn(Fy, -e.gy); Fz = __fadd_rn(Fz, -e.gz);
        });
    });
    const float4 u_before = u;
    const unsigned mode = mass_update(u, v, Fx, Fy, Fz, c);
    if (a.rec_u) {                              // record for the adjoint's reverse sweep
        a.rec_u[mo + cidx] = make_float4(u_before.x, u_before.y, u_before.z, __uint_as_float(mode));
        a.rec_f[mo + cidx] = make_float2(Fx, Fy);
    }
    a.u_out[mo + cidx] = u;
    a.v_out[mo + cidx] = v;
}

}  // namespace

cudaError_t launch_step_streamed(const StreamArgs& a, int n, int max_corners, cudaStream_t s)
{
    if (a.n_robots == 0) return cudaSuccess;
    dim3 grid((max_corners + kStreamThreads - 1) / kStreamThreads, a.n_robots);
    if (a.cube40) k_step_streamed<40><<<grid, kStreamThreads, 0, s>>>(a, n);
    else k_step_streamed<0><<<grid, kStreamThreads, 0, s>>>(a, n);
    return cudaGetLastError();
}

}  // namespace vx
