// Lattice-gather time stepping: the deterministic, atomic-free resident path (Section II-C:
// spring updates then mass updates each step; Table II constants).
//
// A robot's masses sit on the corners of its voxel grid, and every spring joins a corner to one
// of its 13 "forward" lattice neighbours (offset d with a larger corner id).  Each thread owns
// one corner for the whole call and keeps in registers its displacement u, velocity v and the
// (k, alpha L0, beta L0) of its up-to-13 forward springs.  Per step:
//   phase A: for each forward spring (c, c + off(d)) the owner computes the force f from its own
//            u and the neighbour's u (shared memory), adds f to its own total and writes f to
//            the force plane d of shared memory at index c;
//   phase B: each thread subtracts the plane-d entries at c - off(d) of its backward springs, then
//            applies gravity, ground contact with friction and the semi-implicit Euler update in
//            registers and publishes its new u.
// Two block barriers per step, no atomics, and a fixed summation order (own forward springs by
// direction, then backward springs by direction): bit-reproducible.
// Shared memory per robot slot: u and v (float4 per corner) + 13 float4 force planes.
// The state is the displacement from the rest lattice (rest height z0 in u.w), so a spring
// vector is d0 + (u_b - u_a) with d0 the exact lattice offset and the extension is formed without
// cancellation: l - L0 = (2 d0.du + du.du) / (l + L0).
#include "common.cuh"
#include "physics.cuh"

namespace vx {
namespace {

constexpr int kMaxLatticeThreads = 768;
// Polls of a segment's wait on its item's previous segment (each with a 256 ns sleep) before it
// gives up: a few seconds, far beyond any segment's duration.
constexpr uint32_t kSegSpinLimit = 1u << 22;

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// DAMPED: spring dashpots of the paper's preset (a separate instantiation, so the undamped path
// keeps its registers).  RECORD: the adjoint's replay of a checkpoint segment, which also writes
// every step's state before the update with its contact mode, and the horizontal spring force
// before contact.
// SPLIT (with dashpots): split items (item.w == 2: one robot of up to 384 corners alone in a
// block, when the population leaves SMs idle) give every corner a second thread in another warp: the owner evaluates
// directions 0..6, the helper directions 7..12 (writing their planes only), and after the
// barrier the owner adds the helper's six plane entries in direction order before the backward
// gather, so the sums are formed in the same order from the same values: the same bits as the
// unsplit step, with the longest chain of spring evaluations per step cut from 13 to 7.
// IMPOSE: some robots take their contact modes from a table (sim_impose_contact_modes).
// CUBE8: every item of the launch is one 8 x 8 x 8 robot in a 768-thread slot (the MLP
// population's fixed grid); the strides and the plane stride become compile-time constants, so
// the shared-memory addresses of the 13 directions are immediate offsets.
template <bool DAMPED, bool RECORD, bool SPLIT, bool IMPOSE, bool CUBE8 = false>
__global__ void __launch_bounds__(kMaxLatticeThreads, 1) k_step_lattice(LatticeArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    __shared__ int sh_item[5];
    const int tid = threadIdx.x;
    const StepConst c = a.c;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(a.queue, 1);
            if (it < a.n_items) {
                const int4 item = a.items[it];
                sh_item[0] = item.x; sh_item[1] = item.y; sh_item[2] = item.z; sh_item[3] = 1;
                sh_item[4] = item.w;
            } else {
                sh_item[3] = 0;
            }
        }
        __syncthreads();
        if (!sh_item[3]) break;
        const int first = sh_item[0], count = sh_item[1], gthreads = sh_item[2];
        // split groups only in the SPLIT instantiation (launched when the plan has some); the
        // other instantiations run a split item as one unsplit group of 2 S threads
        const bool split = SPLIT && sh_item[4] == 2;
        const int group = CUBE8 ? 0 : tid / gthreads, lt = CUBE8 ? tid : tid % gthreads;
        __syncthreads();   // everyone has read the item before thread 0 may overwrite it
        if (group < count) {
            const int r = a.item_robots[first + group];
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
            const int X = CUBE8 ? 9 : nx + 1, XY = CUBE8 ? 81 : (nx + 1) * (ny + 1), C = CUBE8 ? 729 : XY * (nz + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            // shared-memory slot of this group (S corners): u, then 13 force planes; a split
            // group has 2 S threads, owners [0, S) and helpers [S, 2 S) (whole warps each)
            const int S = CUBE8 ? kMaxLatticeThreads : (split ? gthreads / 2 : gthreads);
            const bool hlp = split && lt >= S;
            const int li = hlp ? lt - S : lt;
            float4* su = sm4 + (size_t)group * kLatticeSlotVec4 * S;
            float4* sv = su + S;               // velocities (read by spring dashpots)
            float4* fb = sv + S;               // plane d at fb + d * S: force on a of spring (a, d)
            // thread li owns the li-th mass (ascending corner order: neighbouring threads touch
            // neighbouring shared-memory rows); threads past the mass count only take part in the
            // barriers
            const int M = a.pv.n_mass[r];
            const bool in = li < M;
            const int cidx = in ? a.corner_order[mo + li] : 0;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            float pk[13], pa[13], pb[13];
            const float* prm = a.prm + 39 * mo;
            for_each_dir([&](auto t) {
                constexpr int d = decltype(t)::value;
                const bool has = ((fl >> d) & 1u) && (!split || hlp == (d >= 7));
                pk[d] = has ? prm[(0 * 13 + d) * C + cidx] : 0.f;
                pa[d] = has ? prm[(1 * 13 + d) * C + cidx] : 0.f;
                pb[d] = has ? prm[(2 * 13 + d) * C + cidx] : 0.f;
            });
            float4 u = in ? a.u[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v = in ? a.v[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            const bool mass = ((fl >> 31) & 1u) && !hlp;
            const int64_t imp = IMPOSE ? a.imp_off[r] : -1;
            if (in && !hlp) {
                su[cidx] = u;
                if (DAMPED) sv[cidx] = v;
            }
            group_sync(bar, gthreads);
            for (int n = 0; n < a.nsteps; ++n) {
                if (hlp && in) {                   // the owner's state after the previous step
                    u = su[cidx];
                    if (DAMPED) v = sv[cidx];
                }
                if (a.ckpt_u && in && !hlp && n % a.ckpt_every == 0) {   // state at the start of segment n / K
                    const int64_t o = (int64_t)(n / a.ckpt_every) * a.ckpt_stride + mo + cidx;
                    a.ckpt_u[o] = u;
                    a.ckpt_v[o] = v;
                }
                const float2 sc = a.sc[n];
                float2 Fxy = make_float2(0.f, 0.f);
                float Fz = 0.f;
                // phase A: forward springs (c, c + offset(d)).  No branch per direction: an
                // absent spring has zero parameters and takes the corner itself as its far end
                // (du = 0, so ext = 0 and the force is an exact zero that leaves the sums' bits
                // unchanged); its plane entry is never read.  6.5 % faster than skipping it, and
                // 2.6 % more with the far end's load predicated off (u from the register).
                if (in) for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (split && hlp != (d >= 7)) return;   // the other thread's direction
                    const bool has = (fl >> d) & 1u;
                    if constexpr (DAMPED) {
                        // with dashpots an absent spring would also load a velocity and take a
                        // square root: here the branch is cheaper (17 % on 5x5x5 robots)
                        if (!has) return;
                    }
                    float4 ub = u;
                    if (has) ub = su[cidx + lattice_offset<d>(X, XY)];
                    SpringEval e = spring_eval_ends<d>(ub, u, c.edge, lattice_rest<d>(c), lattice_rest_sq<d>(c),
                                                      pk[d], pa[d], pb[d], sc.x, sc.y);
                    if constexpr (DAMPED) {
                        const float4 vb = sv[has ? cidx + lattice_offset<d>(X, XY) : cidx];
                        spring_dashpot(e, __fsub_rn(vb.x, v.x), __fsub_rn(vb.y, v.y), __fsub_rn(vb.z, v.z), pk[d], c);
                    }
                    Fxy = __fadd2_rn(Fxy, make_float2(e.gx, e.gy)); Fz = __fadd_rn(Fz, e.gz);
                    // the plane's fourth lane is never read: it takes a value already in a
                    // register (the extension) rather than a zero (2.3 % fewer instructions)
                    fb[d * S + cidx] = make_float4(e.gx, e.gy, e.gz, e.ext);
                });
                group_sync(bar, gthreads);
                // phase B (owners): the helper's forward springs in direction order, then the
                // backward springs (c - offset(d), c), then the mass update
                if (split && in && !hlp) for_each_dir_in<7, 6>([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> d) & 1u)) return;
                    const float4 g = fb[d * S + cidx];
                    Fxy = __fadd2_rn(Fxy, make_float2(g.x, g.y)); Fz = __fadd_rn(Fz, g.z);
                });
                if (!hlp) for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> (16 + d)) & 1u)) return;
                    const float4 g = fb[d * S + cidx - lattice_offset<d>(X, XY)];   // force on a
                    Fxy = __ffma2_rn(make_float2(g.x, g.y), kMinusOne2, Fxy); Fz = __fsub_rn(Fz, g.z);
                });
                if (mass) {
                    int forced = -1;
                    if constexpr (IMPOSE) {
                        const int64_t gstep = a.imp_step0 + n;
                        if (imp >= 0 && gstep < a.imp_n) forced = a.imp_modes[imp + gstep * C + cidx];
                    }
                    if constexpr (RECORD) {            // replay for the adjoint: the step's inputs
                        const float4 ub4 = u;
                        const unsigned mode = IMPOSE ? mass_update_imposed(u, v, Fxy.x, Fxy.y, Fz, c, forced)
                                                     : mass_update(u, v, Fxy.x, Fxy.y, Fz, c);
                        const int64_t o = (int64_t)n * a.rec_stride + mo + cidx;
                        a.rec_u[o] = make_float4(ub4.x, ub4.y, ub4.z, __uint_as_float(mode));
                        a.rec_f[o] = Fxy;
                    } else if constexpr (IMPOSE) {
                        mass_update_imposed(u, v, Fxy.x, Fxy.y, Fz, c, forced);
                    } else {
                        mass_update(u, v, Fxy.x, Fxy.y, Fz, c);
                    }
                    su[cidx] = u;
                    if (DAMPED) sv[cidx] = v;
                }
                group_sync(bar, gthreads);
            }
            if (in && !hlp) {
                a.u[mo + cidx] = u;
                a.v[mo + cidx] = v;
            }
        }
        __syncthreads();
    }
}


// ----------------------------------------------------------------------------------------------
// Segmented queue for the per-corner step (undamped, no split items, no imposed modes; RECORD as
// above; CUBE8 as above).  With more items than SMs a queue of whole items leaves SMs idle while
// the last wave's robots run all their steps; here every item's steps are cut into a.nseg
// segments of a.seg_steps and the queue holds the (segment, item) units in segment-major order,
// so the last wave waits for one segment.  A unit first waits (thread 0, bounded) until its item's
// previous segment has published progress[item]: that unit lies n_items places earlier in the
// queue and was taken by a running block, so the wait is normally over before it starts, and it
// cannot deadlock (every unit's dependency sits earlier in the queue).  The state passes between
// segments through global memory (stored, fenced, then published; read through L2 after the
// acquire), and every step is the per-corner kernel's arithmetic in its order: the same bits as
// one unit per item (tested).  A separate kernel rather than a template switch of the one above:
// with the switch, the unsegmented instantiations measured 2 % slower.
// ----------------------------------------------------------------------------------------------
template <bool RECORD, bool CUBE8>
__global__ void __launch_bounds__(kMaxLatticeThreads, 1) k_step_lattice_seg(LatticeArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    // item (first robot, robots, threads), more work, -, segment, item index, segment's end
    __shared__ int sh_item[8];
    const int tid = threadIdx.x;
    const StepConst c = a.c;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(a.queue, 1);
            if (it < a.n_items * a.nseg) {
                const int seg = it / a.n_items, ii = it - seg * a.n_items;
                const int4 item = a.items[ii];
                sh_item[0] = item.x; sh_item[1] = item.y; sh_item[2] = item.z; sh_item[3] = 1;
                sh_item[5] = seg; sh_item[6] = ii;
                sh_item[7] = min((seg + 1) * a.seg_steps, a.nsteps);
                if (seg > 0) {
                    uint32_t k = 0;
                    while (ld_acquire_gpu(a.progress + ii) < seg) {
                        if (++k >= kSegSpinLimit) { atomicOr(a.status, 8); break; }
                        __nanosleep(256);
                    }
                }
            } else {
                sh_item[3] = 0;
            }
        }
        __syncthreads();
        if (!sh_item[3]) break;
        const int first = sh_item[0], count = sh_item[1], gthreads = sh_item[2];
        const int n_begin = sh_item[5] * a.seg_steps;
        const int group = CUBE8 ? 0 : tid / gthreads, lt = CUBE8 ? tid : tid % gthreads;
        __syncthreads();   // everyone has read the item before thread 0 may overwrite it
        if (group < count) {
            const int r = a.item_robots[first + group];
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
            const int X = CUBE8 ? 9 : nx + 1, XY = CUBE8 ? 81 : (nx + 1) * (ny + 1), C = CUBE8 ? 729 : XY * (nz + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            const int S = CUBE8 ? kMaxLatticeThreads : gthreads;   // (a split item: one group of 2 S)
            float4* su = sm4 + (size_t)group * kLatticeSlotVec4 * S;
            float4* fb = su + 2 * S;           // plane d at fb + d * S (after u and the unused v)
            const int M = a.pv.n_mass[r];
            const bool in = lt < M;
            const int cidx = in ? a.corner_order[mo + lt] : 0;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            float pk[13], pa[13], pb[13];
            const float* prm = a.prm + 39 * mo;
            for_each_dir([&](auto t) {
                constexpr int d = decltype(t)::value;
                const bool has = (fl >> d) & 1u;
                pk[d] = has ? prm[(0 * 13 + d) * C + cidx] : 0.f;
                pa[d] = has ? prm[(1 * 13 + d) * C + cidx] : 0.f;
                pb[d] = has ? prm[(2 * 13 + d) * C + cidx] : 0.f;
            });
            // the previous segment's state, written by another SM: read through L2
            float4 u = in ? __ldcg(a.u + mo + cidx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v = in ? __ldcg(a.v + mo + cidx) : make_float4(0.f, 0.f, 0.f, 0.f);
            const bool mass = (fl >> 31) & 1u;
            if (in) su[cidx] = u;
            group_sync(bar, gthreads);
            // (the segment's end is re-read from shared memory each step rather than held in a
            // register through the step)
            for (int n = n_begin; n < *(volatile int*)&sh_item[7]; ++n) {
                if (a.ckpt_u && in && n % a.ckpt_every == 0) {   // state at the start of segment n / K
                    const int64_t o = (int64_t)(n / a.ckpt_every) * a.ckpt_stride + mo + cidx;
                    a.ckpt_u[o] = u;
                    a.ckpt_v[o] = v;
                }
                const float2 sc = a.sc[n];
                float2 Fxy = make_float2(0.f, 0.f);
                float Fz = 0.f;
                // phase A: forward springs, branch-free (an absent spring is an exact zero force)
                if (in) for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    const bool has = (fl >> d) & 1u;
                    float4 ub = u;
                    if (has) ub = su[cidx + lattice_offset<d>(X, XY)];
                    SpringEval e = spring_eval_ends<d>(ub, u, c.edge, lattice_rest<d>(c), lattice_rest_sq<d>(c),
                                                      pk[d], pa[d], pb[d], sc.x, sc.y);
                    Fxy = __fadd2_rn(Fxy, make_float2(e.gx, e.gy)); Fz = __fadd_rn(Fz, e.gz);
                    fb[d * S + cidx] = make_float4(e.gx, e.gy, e.gz, e.ext);
                });
                group_sync(bar, gthreads);
                // phase B: backward springs in direction order, then the mass update
                if (in) for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((fl >> (16 + d)) & 1u)) return;
                    const float4 g = fb[d * S + cidx - lattice_offset<d>(X, XY)];   // force on a
                    Fxy = __ffma2_rn(make_float2(g.x, g.y), kMinusOne2, Fxy); Fz = __fsub_rn(Fz, g.z);
                });
                if (mass) {
                    if constexpr (RECORD) {            // the step's inputs, for the adjoint
                        const float4 ub4 = u;
                        const unsigned mode = mass_update(u, v, Fxy.x, Fxy.y, Fz, c);
                        const int64_t o = (int64_t)n * a.rec_stride + mo + cidx;
                        a.rec_u[o] = make_float4(ub4.x, ub4.y, ub4.z, __uint_as_float(mode));
                        a.rec_f[o] = Fxy;
                    } else {
                        mass_update(u, v, Fxy.x, Fxy.y, Fz, c);
                    }
                    su[cidx] = u;
                }
                group_sync(bar, gthreads);
            }
            if (in) {
                a.u[mo + cidx] = u;
                a.v[mo + cidx] = v;
                __threadfence();                   // visible before the segment is published
            }
        }
        __syncthreads();
        if (tid == 0) st_release_gpu(a.progress + sh_item[6], sh_item[5] + 1);
    }
}


// ----------------------------------------------------------------------------------------------
// Direction-compacted variant of the same step.  In the per-corner kernel above a warp spends an
// evaluation on direction d whenever any of its 32 corners has a spring along d, so partly
// filled grids pay for absent springs.  Here thread t's slot d holds the t-th existing spring of
// direction d (the direction-major packed list), so along every direction the busy threads are
// 0 .. n_d - 1 and whole warps past n_d skip it: the cost of phase A follows the spring count.
// Per step:
//   phase A: slot d of every thread below n_d evaluates its spring (a, a + off(d)) from the shared
//            positions and writes the force on a to plane d at index a;
//   phase B: each mass thread adds its forward planes (index c) and subtracts its backward planes
//            (index c - off(d)) in direction order, then the mass update.
// Same arithmetic (compile-time directions), same per-mass summation order (forward by direction,
// then backward by direction) and same initial zero as the per-corner kernel: the two give
// identical bits.  It trades instructions for shared-memory traffic (phase A also reads u_a and
// phase B also reads the forward planes).
// ----------------------------------------------------------------------------------------------
template <bool DAMPED>
__global__ void __launch_bounds__(kMaxLatticeThreads, 1) k_step_lattice_compact(LatticeArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    __shared__ int sh_item[4];
    __shared__ int sh_nd[kMaxLatticeThreads / 64][16];   // per group: springs per direction
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
        __syncthreads();
        if (group < count) {
            const int r = a.item_robots[first + group];
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1];
            const int X = nx + 1, XY = (nx + 1) * (ny + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            const int S = gthreads;
            float4* su = sm4 + (size_t)group * kLatticeSlotVec4 * S;
            float4* sv = su + S;
            float4* fb = sv + S;
            int* nd = sh_nd[group];
            const int M = a.pv.n_mass[r];
            const bool in = lt < M;
            const int cidx = in ? a.corner_order[mo + lt] : 0;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            // springs per direction = corners with that forward bit
            if (lt < 13) nd[lt] = 0;
            group_sync(bar, gthreads);
            for_each_dir([&](auto t) {
                constexpr int d = decltype(t)::value;
                const unsigned w = __ballot_sync(0xffffffffu, (fl >> d) & 1u);
                if ((lt & 31) == 0 && w) atomicAdd(&nd[d], __popc(w));
            });
            group_sync(bar, gthreads);
            // slot d: the lt-th spring of direction d, at list offset (springs of directions < d) + lt
            const float4* __restrict__ list = a.spack + a.pv.soff[r];
            float pk[13], pa[13], pb[13];
            uint32_t cpack[5];                                     // the slots' corners a, 10 bits each
            uint32_t has = 0u;
#pragma unroll
            for (int i = 0; i < 5; ++i) cpack[i] = 0u;
            int base = 0;
            for_each_dir([&](auto t) {
                constexpr int d = decltype(t)::value;
                const int n_d = nd[d];
                const bool h = lt < n_d;
                const float4 p = h ? list[base + lt] : make_float4(0.f, 0.f, 0.f, 0.f);
                pk[d] = p.x; pa[d] = p.y; pb[d] = p.z;
                cpack[d / 3] |= (__float_as_uint(p.w) & 0x3ffu) << (10 * (d % 3));
                has |= (h ? 1u : 0u) << d;
                base += n_d;
            });
            float4 u = in ? a.u[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v = in ? a.v[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) {
                su[cidx] = u;
                if (DAMPED) sv[cidx] = v;
            }
            group_sync(bar, gthreads);
            for (int n = 0; n < a.nsteps; ++n) {
                if (a.ckpt_u && in && n % a.ckpt_every == 0) {
                    const int64_t o = (int64_t)(n / a.ckpt_every) * a.ckpt_stride + mo + cidx;
                    a.ckpt_u[o] = u;
                    a.ckpt_v[o] = v;
                }
                const float2 sc = a.sc[n];
                // phase A: this thread's slot of every direction.  The corner words are re-read
                // as opaque values every step so the compiler decodes them where used instead of
                // keeping 13 decoded corners (and their neighbours) live across the loop.
#pragma unroll
                for (int i = 0; i < 5; ++i) asm volatile("" : "+r"(cpack[i]));
                asm volatile("" : "+r"(has));
                for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    if (!((has >> d) & 1u)) return;
                    const int ca = (int)((cpack[d / 3] >> (10 * (d % 3))) & 0x3ffu);
                    const int cb = ca + lattice_offset<d>(X, XY);
                    const float4 ua = su[ca];
                    const float4 ub = su[cb];
                    SpringEval e = spring_eval_ends<d>(ub, ua, c.edge, lattice_rest<d>(c), lattice_rest_sq<d>(c),
                                                      pk[d], pa[d], pb[d], sc.x, sc.y);
                    if constexpr (DAMPED) {
                        const float4 va = sv[ca];
                        const float4 vb = sv[cb];
                        spring_dashpot(e, __fsub_rn(vb.x, va.x), __fsub_rn(vb.y, va.y), __fsub_rn(vb.z, va.z), pk[d], c);
                    }
                    fb[d * S + ca] = make_float4(e.gx, e.gy, e.gz, e.ext);
                });
                group_sync(bar, gthreads);
                // phase B: the forces of this mass's springs in direction order, then the update
                if (in) {
                    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
                    for_each_dir([&](auto t) {
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> d) & 1u)) return;
                        const float4 g = fb[d * S + cidx];
                        Fx = __fadd_rn(Fx, g.x); Fy = __fadd_rn(Fy, g.y); Fz = __fadd_rn(Fz, g.z);
                    });
                    for_each_dir([&](auto t) {
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> (16 + d)) & 1u)) return;
                        const float4 g = fb[d * S + cidx - lattice_offset<d>(X, XY)];
                        Fx = __fsub_rn(Fx, g.x); Fy = __fsub_rn(Fy, g.y); Fz = __fsub_rn(Fz, g.z);
                    });
                    mass_update(u, v, Fx, Fy, Fz, c);
                    su[cidx] = u;
                    if (DAMPED) sv[cidx] = v;
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

// ----------------------------------------------------------------------------------------------
// Mass-packed variant of the per-corner step.  The kernel above gives every robot a slot sized
// by its grid corners, and threads past the robot's mass count only join the barriers: an
// evolved 8x8x8 robot of ~400 masses leaves half of a 768-thread block idle.  Here a block's
// 768 threads are shared by several robots, each group sized by its mass count (a multiple of
// 32 threads), so a block runs as many masses as it has threads.  What makes that fit in shared
// memory is indexing the force planes by the thread slot of the spring's far end (the reader)
// instead of by corner: a robot needs 13 planes of T entries (T = its threads) and its
// displacements by corner (C entries), not 13 planes of C entries.  The far end's slot rides in
// the .w lane of its shared displacement, which the spring evaluation loads anyway.
// Per step:
//   phase A: for each forward spring (c, c + off(d)) the owner computes the force f from its own
//            displacement and the far end's, adds f to its own total, and writes f into plane d
//            at the far end's slot (absent springs write a never-read row per lane);
//   phase B: each thread subtracts the plane-d entries at its own slot for its backward springs
//            (contiguous, conflict-free rows), then the mass update.
// The sums run over the same values in the same order as the per-corner kernel (own forward
// springs by direction, then backward springs by direction): identical bits, so the adjoint's
// replay (which runs the per-corner kernel) reproduces a run of this one.
// Shared memory of a group: C float4 displacements (+ C velocities with dashpots), 13 T float4
// plane entries, 32 float4 rows for absent springs.
// ----------------------------------------------------------------------------------------------
template <bool DAMPED>
__global__ void __launch_bounds__(kMaxLatticeThreads, 1) k_step_lattice_packed(LatticeArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    __shared__ int sh_item[3];
    const int tid = threadIdx.x;
    const StepConst c = a.c;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(a.queue, 1);
            if (it < a.n_items) {
                const int4 item = a.items[it];
                sh_item[0] = item.x; sh_item[1] = item.y; sh_item[2] = 1;
            } else {
                sh_item[2] = 0;
            }
        }
        __syncthreads();
        if (!sh_item[2]) break;
        const int first = sh_item[0], count = sh_item[1];
        __syncthreads();   // everyone has read the item before thread 0 may overwrite it
        // this thread's group: the one whose thread range [t0, t0 + T) holds it (groups are
        // whole warps; threads past the last group only wait for the next item)
        int group = -1;
        int4 gi = make_int4(0, 0, 0, 0);
        for (int j = 0; j < count; ++j) {
            const int4 q = a.groups[first + j];
            if (tid >= q.y && tid < q.y + q.z) { group = j; gi = q; }
        }
        if (group >= 0) {
            const int r = gi.x, T = gi.z, lt = tid - gi.y;
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
            const int X = nx + 1, XY = (nx + 1) * (ny + 1), C = XY * (nz + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            float4* su = sm4 + gi.w;                 // displacements by corner, slot id in .w
            float4* sv = su + C;                     // velocities by corner (dashpots only)
            float4* fb = DAMPED ? sv + C : su + C;   // plane d at fb + d * T, by the reader's slot;
                                                     // then 32 rows for absent springs (never read)
            const int M = a.pv.n_mass[r];
            const bool in = lt < M;
            const int cidx = in ? a.corner_order[mo + lt] : 0;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            const float slot = __int_as_float(lt);
            const int junk = 13 * T + (lt & 31);     // this lane's row for absent springs
            float pk[13], pa[13], pb[13];
            const float* prm = a.prm + 39 * mo;
            for_each_dir([&](auto t) {
                constexpr int d = decltype(t)::value;
                const bool has = (fl >> d) & 1u;
                pk[d] = has ? prm[(0 * 13 + d) * C + cidx] : 0.f;
                pa[d] = has ? prm[(1 * 13 + d) * C + cidx] : 0.f;
                pb[d] = has ? prm[(2 * 13 + d) * C + cidx] : 0.f;
            });
            float4 u = in ? a.u[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v = in ? a.v[mo + cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) {
                su[cidx] = make_float4(u.x, u.y, u.z, slot);
                if (DAMPED) sv[cidx] = v;
            }
            group_sync(bar, T);
            for (int n = 0; n < a.nsteps; ++n) {
                if (a.ckpt_u && in && n % a.ckpt_every == 0) {   // state at the start of segment n / K
                    const int64_t o = (int64_t)(n / a.ckpt_every) * a.ckpt_stride + mo + cidx;
                    a.ckpt_u[o] = u;
                    a.ckpt_v[o] = v;
                }
                const float2 sc = a.sc[n];
                float2 Fxy = make_float2(0.f, 0.f);
                float Fz = 0.f;
                // phase A: forward springs, no branch per direction (an absent spring has zero
                // parameters and the corner itself as far end: an exact zero force)
                if (in) for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    const bool has = (fl >> d) & 1u;
                    if constexpr (DAMPED) {
                        if (!has) return;
                    }
                    float4 ub = u;
                    if (has) ub = su[cidx + lattice_offset<d>(X, XY)];
                    SpringEval e = spring_eval_ends<d>(ub, u, c.edge, lattice_rest<d>(c), lattice_rest_sq<d>(c),
                                                      pk[d], pa[d], pb[d], sc.x, sc.y);
                    if constexpr (DAMPED) {
                        const float4 vb = sv[cidx + lattice_offset<d>(X, XY)];
                        spring_dashpot(e, __fsub_rn(vb.x, v.x), __fsub_rn(vb.y, v.y), __fsub_rn(vb.z, v.z), pk[d], c);
                    }
                    Fxy = __fadd2_rn(Fxy, make_float2(e.gx, e.gy)); Fz = __fadd_rn(Fz, e.gz);
                    const int row = has ? d * T + __float_as_int(ub.w) : junk;
                    fb[row] = make_float4(e.gx, e.gy, e.gz, e.ext);
                });
                group_sync(bar, T);
                // phase B: backward springs (c - offset(d), c) from this slot's rows, then the update
                if (in) {
                    for_each_dir([&](auto t) {
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> (16 + d)) & 1u)) return;
                        const float4 g = fb[d * T + lt];   // force on the spring's first end
                        Fxy = __ffma2_rn(make_float2(g.x, g.y), kMinusOne2, Fxy); Fz = __fsub_rn(Fz, g.z);
                    });
                    if ((fl >> 31) & 1u) {
                        mass_update(u, v, Fxy.x, Fxy.y, Fz, c);
                        su[cidx] = make_float4(u.x, u.y, u.z, slot);
                        if (DAMPED) sv[cidx] = v;
                    }
                }
                group_sync(bar, T);
            }
            if (in) {
                a.u[mo + cidx] = u;
                a.v[mo + cidx] = v;
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------------------------
// Segmented queue for the mass-packed step (undamped): the packed items' steps cut into a.nseg
// segments, queued segment-major, each unit waiting (bounded) for its item's previous segment
// and publishing its own, exactly as k_step_lattice_seg does for the per-corner step; the step
// itself is k_step_lattice_packed's undamped arithmetic in its order (the same bits as whole runs).
// ----------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kMaxLatticeThreads, 1) k_step_lattice_packed_seg(LatticeArgs a)
{
    extern __shared__ __align__(16) float4 sm4[];
    // item (first group, groups), more work, -, -, segment, item index, segment's end
    __shared__ int sh_item[8];
    const int tid = threadIdx.x;
    const StepConst c = a.c;
    for (;;) {
        if (tid == 0) {
            const int it = atomicAdd(a.queue, 1);
            if (it < a.n_items * a.nseg) {
                const int seg = it / a.n_items, ii = it - seg * a.n_items;
                const int4 item = a.items[ii];
                sh_item[0] = item.x; sh_item[1] = item.y; sh_item[2] = 1;
                sh_item[5] = seg; sh_item[6] = ii;
                sh_item[7] = min((seg + 1) * a.seg_steps, a.nsteps);
                if (seg > 0) {
                    uint32_t k = 0;
                    while (ld_acquire_gpu(a.progress + ii) < seg) {
                        if (++k >= kSegSpinLimit) { atomicOr(a.status, 8); break; }
                        __nanosleep(256);
                    }
                }
            } else {
                sh_item[2] = 0;
            }
        }
        __syncthreads();
        if (!sh_item[2]) break;
        const int first = sh_item[0], count = sh_item[1];
        const int n_begin = sh_item[5] * a.seg_steps;
        __syncthreads();   // everyone has read the item before thread 0 may overwrite it
        int group = -1;
        int4 gi = make_int4(0, 0, 0, 0);
        for (int j = 0; j < count; ++j) {
            const int4 q = a.groups[first + j];
            if (tid >= q.y && tid < q.y + q.z) { group = j; gi = q; }
        }
        if (group >= 0) {
            const int r = gi.x, T = gi.z, lt = tid - gi.y;
            const int nx = a.pv.dims[3 * r], ny = a.pv.dims[3 * r + 1], nz = a.pv.dims[3 * r + 2];
            const int X = nx + 1, XY = (nx + 1) * (ny + 1), C = XY * (nz + 1);
            const int64_t mo = a.pv.moff[r];
            const int bar = 1 + group;
            float4* su = sm4 + gi.w;                 // displacements by corner, slot id in .w
            float4* fb = su + C;                     // plane d at fb + d * T, by the reader's slot;
                                                     // then 32 rows for absent springs (never read)
            const int M = a.pv.n_mass[r];
            const bool in = lt < M;
            const int cidx = in ? a.corner_order[mo + lt] : 0;
            const uint32_t fl = in ? a.cflags[mo + cidx] : 0u;
            const float slot = __int_as_float(lt);
            const int junk = 13 * T + (lt & 31);     // this lane's row for absent springs
            float pk[13], pa[13], pb[13];
            const float* prm = a.prm + 39 * mo;
            for_each_dir([&](auto t) {
                constexpr int d = decltype(t)::value;
                const bool has = (fl >> d) & 1u;
                pk[d] = has ? prm[(0 * 13 + d) * C + cidx] : 0.f;
                pa[d] = has ? prm[(1 * 13 + d) * C + cidx] : 0.f;
                pb[d] = has ? prm[(2 * 13 + d) * C + cidx] : 0.f;
            });
            // the previous segment's state, written by another SM: read through L2
            float4 u = in ? __ldcg(a.u + mo + cidx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v = in ? __ldcg(a.v + mo + cidx) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) su[cidx] = make_float4(u.x, u.y, u.z, slot);
            group_sync(bar, T);
            for (int n = n_begin; n < *(volatile int*)&sh_item[7]; ++n) {
                if (a.ckpt_u && in && n % a.ckpt_every == 0) {   // state at the start of segment n / K
                    const int64_t o = (int64_t)(n / a.ckpt_every) * a.ckpt_stride + mo + cidx;
                    a.ckpt_u[o] = u;
                    a.ckpt_v[o] = v;
                }
                const float2 sc = a.sc[n];
                float2 Fxy = make_float2(0.f, 0.f);
                float Fz = 0.f;
                if (in) for_each_dir([&](auto t) {
                    constexpr int d = decltype(t)::value;
                    const bool has = (fl >> d) & 1u;
                    float4 ub = u;
                    if (has) ub = su[cidx + lattice_offset<d>(X, XY)];
                    SpringEval e = spring_eval_ends<d>(ub, u, c.edge, lattice_rest<d>(c), lattice_rest_sq<d>(c),
                                                      pk[d], pa[d], pb[d], sc.x, sc.y);
                    Fxy = __fadd2_rn(Fxy, make_float2(e.gx, e.gy)); Fz = __fadd_rn(Fz, e.gz);
                    const int row = has ? d * T + __float_as_int(ub.w) : junk;
                    fb[row] = make_float4(e.gx, e.gy, e.gz, e.ext);
                });
                group_sync(bar, T);
                if (in) {
                    for_each_dir([&](auto t) {
                        constexpr int d = decltype(t)::value;
                        if (!((fl >> (16 + d)) & 1u)) return;
                        const float4 g = fb[d * T + lt];   // force on the spring's first end
                        Fxy = __ffma2_rn(make_float2(g.x, g.y), kMinusOne2, Fxy); Fz = __fsub_rn(Fz, g.z);
                    });
                    if ((fl >> 31) & 1u) {
                        mass_update(u, v, Fxy.x, Fxy.y, Fz, c);
                        su[cidx] = make_float4(u.x, u.y, u.z, slot);
                    }
                }
                group_sync(bar, T);
            }
            if (in) {
                a.u[mo + cidx] = u;
                a.v[mo + cidx] = v;
                __threadfence();                   // visible before the segment is published
            }
        }
        __syncthreads();
        if (tid == 0) st_release_gpu(a.progress + sh_item[6], sh_item[5] + 1);
    }
}

}  // namespace

int lattice_max_threads() { return kMaxLatticeThreads; }

cudaError_t launch_step_lattice_packed(const LatticeArgs& a, int grid, size_t smem, cudaStream_t s)
{
    // a segmented queue (a.nseg > 1; the host sets it only for undamped robots)
    auto kernel = a.nseg > 1 ? k_step_lattice_packed_seg
                : (a.c.damped ? k_step_lattice_packed<true> : k_step_lattice_packed<false>);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, kMaxLatticeThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_step_lattice(const LatticeArgs& a, int grid, int threads, size_t smem,
                                cudaStream_t s)
{
    const bool cube8 = a.cube8 && !a.c.damped;
    // a segmented queue (a.nseg > 1; the host sets it only for undamped per-corner items without
    // imposed modes, recording only on 8 x 8 x 8 robots)
    if (a.nseg > 1) {
        auto kseg = a.rec_u ? k_step_lattice_seg<true, true>
                  : (cube8 ? k_step_lattice_seg<false, true> : k_step_lattice_seg<false, false>);
        cudaError_t e = cudaFuncSetAttribute(kseg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kseg<<<grid, threads, smem, s>>>(a);
        return cudaGetLastError();
    }
    auto kernel = a.imp_modes ? (a.rec_u ? k_step_lattice<false, true, false, true> : k_step_lattice<false, false, false, true>)
                : a.rec_u ? (cube8 ? k_step_lattice<false, true, false, false, true> : k_step_lattice<false, true, false, false>)
                : (cube8 && !a.spack) ? k_step_lattice<false, false, false, false, true>
                : a.spack ? (a.c.damped ? k_step_lattice_compact<true> : k_step_lattice_compact<false>)
                : a.c.damped ? (a.has_split ? k_step_lattice<true, false, true, false> : k_step_lattice<true, false, false, false>)
                             : k_step_lattice<false, false, false, false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vx
