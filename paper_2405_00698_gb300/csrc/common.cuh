// Internal declarations shared by the CUDA translation units of the voxsim library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/voxsim.h"

namespace vx {

// ----------------------------------------------------------------------------------------------
// Constants
// ----------------------------------------------------------------------------------------------
constexpr int kNumMat = 5;
constexpr int kGenome = 20998;       // MLP 3 -> gamma(256) -> 64 -> 64 -> 6
constexpr int kPeRows = 128;         // m of Eq. (1)
constexpr int kPeDim = 256;          // 2m
constexpr int kHidden = 64;
constexpr int kOut = 6;
constexpr int kOffW1 = 0, kOffB1 = 16384, kOffW2 = 16448, kOffB2 = 20544, kOffW3 = 20608,
              kOffB3 = 20992;
constexpr int kMaxAxis = 64;          // largest grid extent per axis
constexpr int kResidentMaxCorner = 16383;  // packed 14-bit corner ids on the resident path

// The 13 lattice directions (dx, dy, dz) of springs from a corner to a larger corner id, in
// increasing (dz, dy, dx) order: (1,0,0) (-1,1,0) (0,1,0) (1,1,0) (-1,-1,1) (0,-1,1) (1,-1,1)
// (-1,0,1) (0,0,1) (1,0,1) (-1,1,1) (0,1,1) (1,1,1).  Component `axis` of direction d, stored
// as 2-bit fields (value + 1); a packed resident spring stores its direction index.
__host__ __device__ constexpr int lattice_dir(int d, int axis)
{
    return (int)((axis == 0 ? 0x2492492u : (axis == 1 ? 0x2a540a9u : 0x2aaaa55u)) >> (2 * d) & 3u) - 1;
}

// Per-material constants in float, passed by value to kernels.
struct MatConst {
    float k[kNumMat];
    float amp[kNumMat];
    float phase[kNumMat];
};

// Physics constants in float for the step kernels.
struct StepConst {
    float dt;
    float dt_over_m;    // dt / mass
    float weight;       // mass * gravity
    float damping;
    // the step constants carried past float32: a float32 dt, dt / m or m g is off by up to 3e-8
    // of itself (0.999 by 1.3e-8), the same in every step, and at 2000 steps such a fixed
    // offset of the map moves its gradients by more than 1e-3 of the largest entry; each is
    // applied as a pair hi + lo (lo = the float32 of the remainder), the damping as
    // c w = w - (1 - c) w with 1 - c in float32 (an error of 1e-11 of c)
    float dt_lo;
    float dtm_lo;
    float weight_lo;
    float damping_c;    // 1 - damping
    float mu_k_lo;
    float k_ground;
    float mu_s;
    float mu_k;
    float edge;
    float edge_sqrt2;
    float edge_sqrt3;
    float edge_sq;      // rest lengths squared: edge^2, 2 edge^2, 3 edge^2
    float edge_sq2;
    float edge_sq3;
    int ground_on;
    int damped;         // spring dashpots present (spring_c > 0)
    float spring_c;     // 2 zeta_s sqrt(mass / 2): dashpot coefficient = spring_c sqrt(k)
    float ground_c;     // 2 zeta_g sqrt(k_ground mass)
};

// Device view of a population's layout.
struct PopView {
    int P;
    const int* dims;         // [3P]
    const int64_t* voff;     // [P+1] voxel offsets
    const int64_t* moff;     // [P+1] mass (= corner) capacity offsets
    const int64_t* soff;     // [P+1] spring capacity offsets
    int* n_mass;             // [P]
    int* n_spring;           // [P]
};

// ----------------------------------------------------------------------------------------------
// Kernel launchers (each returns the launch error, if any)
// ----------------------------------------------------------------------------------------------
cudaError_t launch_decode_materials(const uint8_t* mats, int64_t n, MatConst mc, uint8_t* mat,
                                    float* w, float* kappa, float* phi, int* bad, cudaStream_t s);
cudaError_t launch_decode_logits(const float* logits, int64_t n, MatConst mc, uint8_t* mat,
                                 float* w, float* kappa, float* phi, cudaStream_t s);
cudaError_t launch_decode_params(const uint8_t* mats, const float* w_in, const float* k_in,
                                 const float* p_in, int64_t n, uint8_t* mat, float* w,
                                 float* kappa, float* phi, int* bad, cudaStream_t s);
cudaError_t launch_decode_param_rows(const uint8_t* mats, const float* rows, int64_t V, int64_t n,
                                     uint8_t* mat, float* w, float* kappa, float* phi, int* bad,
                                     cudaStream_t s);
cudaError_t launch_pe_table(int nx, int ny, int nz, const float* B, void* pe_bf16,
                            cudaStream_t s);
cudaError_t launch_grad_step(float* genomes, int G, int64_t V, const int64_t* voff, const float* g_w,
                             const float* g_kappa, const float* g_phi, const int* rows, int n_rows,
                             float eta_w, float eta_kappa, float eta_phi, const float* lo,
                             const float* hi, cudaStream_t s);
cudaError_t launch_mlp_query(int P, int Q, const void* pe_bf16, const float* genomes, MatConst mc,
                             uint8_t* mat, float* w, float* kappa, float* phi, int* status,
                             int num_sms, cudaStream_t s);
size_t mlp_tc_smem_bytes();
cudaError_t launch_mlp_query_simt(int P, int Q, const void* pe_bf16, const float* genomes,
                                  MatConst mc, uint8_t* mat, float* w, float* kappa, float* phi,
                                  cudaStream_t s);

cudaError_t launch_topology(PopView pv, const uint8_t* mat_raw, uint8_t* mat, const float* w,
                            const float* kappa, const float* phi, MatConst mc, double edge,
                            int* label, int* count, int* corner_mass, int* mass_corner,
                            int2* spr_ab, float4* spr_p, float4* spr_pack, uint32_t* cflags,
                            float* prm, float4* x0, float4* x, float4* v, double* x0c, int* status,
                            int max_threads, cudaStream_t s);

cudaError_t launch_sincos_table(double omega, double dt, int64_t step0, int n, float2* out,
                                cudaStream_t s);

struct ResidentArgs {
    PopView pv;
    const float4* spr_pack;  // packed springs (k, alpha L0, beta L0, a | b << 14 | dir << 28),
                             // a and b corner ids
    const uint32_t* cflags;  // per corner: bit 31 set where a mass sits
    float4* x;               // per corner: displacement from the rest lattice, rest height in .w
    float4* v;
    const float2* sc;        // sin / cos of w t per step of this call
    int nsteps;
    StepConst c;
    const int* order;        // robots to process, longest first
    int n_robots;            // entries of order
    int* queue;              // work counter (zeroed by the launcher) or NULL for static split
    int max_mass;            // smem layout: masses per robot slot
    int max_spring_smem;     // springs cached in shared memory per robot (after those in tensor memory)
    int tm_rec;              // springs per thread held in tensor memory (0: none, nothing allocated)
    int tm_cols;             // tensor-memory columns per warp (of the block's 512)
    int accumulate;          // SIM_ACC_ATOMIC or SIM_ACC_GATHER
    // gather path
    const int* inc_off;      // [moff-based] per-mass incidence start (length M+1 per robot)
    const int* inc_list;     // [soff*2-based] spring index * 2 + side
};
cudaError_t launch_step_resident(const ResidentArgs& a, int grid, int threads, size_t smem,
                                 cudaStream_t s);

// Lattice-gather path (deterministic): work items of robots of one size class.
struct LatticeArgs {
    PopView pv;
    const int* corner_order; // per robot at moff: the mass corners (ascending), one per thread
    const uint32_t* cflags;  // per corner: forward mask bits 0..12, backward 16..28, mass bit 31
    const float* prm;        // per robot at 39 * moff: [3][13][C] (k, alpha L0, beta L0)
    // spring-parallel variant (NULL: per-corner variant): the direction-major packed springs
    // per robot at soff, (k, alpha L0, beta L0, a | b << 14 | direction << 28)
    const float4* spack;
    float4* u;               // per corner displacement (rest height in .w)
    float4* v;               // per corner velocity
    const float2* sc;        // sin / cos of w t per step of this call
    int nsteps;
    StepConst c;
    const int4* items;       // (first robot in item_robots, robots, threads per robot, kind:
                             // 0 per corner, 1 direction-compacted, 2 per corner split); for the
                             // mass-packed kernel (first group in groups, groups, 0, 0)
    const int* item_robots;
    const int4* groups;      // mass-packed kernel: per group (robot, first thread, threads,
                             // shared-memory offset in float4)
    int n_items;
    // per-corner kernel, segmented queue (nseg > 1): unit u = seg * n_items + item steps the
    // item's robots through steps [seg * seg_steps, min((seg + 1) * seg_steps, nsteps)) once the
    // item's previous segment has published progress[item] = seg (zeroed before the launch);
    // a wait that gives up sets bit 3 of *status
    int nseg;
    int seg_steps;
    int* progress;
    int* status;
    int has_split;           // the items include split ones (run by the split instantiation)
    int cube8;               // every per-corner item is one 8 x 8 x 8 robot in a 768-thread slot
    int* queue;              // work counter, zeroed before the launch
    // checkpoints for the adjoint (NULL when off): state at steps 0, K, 2K, ... of the call
    float4* ckpt_u;
    float4* ckpt_v;
    int64_t ckpt_stride;     // corners per checkpoint (sum over robots)
    int ckpt_every;          // K
    // replay records for the adjoint (NULL when off; undamped only): per step n of the call, at
    // n * rec_stride + corner, the state before the update (contact mode in .w) and the
    // horizontal spring force before contact
    float4* rec_u;
    float2* rec_f;
    int64_t rec_stride;
    // imposed contact modes (NULL: none; sim_impose_contact_modes): robot r's table of imp_n
    // steps x its C corners at imp_off[r] (-1: the robot decides its modes), indexed by the run
    // step imp_step0 + n of this call's step n
    const uint8_t* imp_modes;
    const int64_t* imp_off;
    int imp_n;
    int64_t imp_step0;
};

// Streamed path (robots too large for one SM): one launch per step over all their corners.
struct StreamArgs {
    PopView pv;
    const uint32_t* cflags;
    const float* prm;
    const float4* u_in;      // positions at the start of the step (per corner)
    float4* u_out;           // positions at its end
    const float4* v_in;      // velocities at the start of the step
    float4* v_out;           // velocities at its end
    const float2* sc;        // sin / cos of w t per step of this call (indexed by the step)
    StepConst c;
    const int* robots;       // streamed robots (grid.y)
    int n_robots;
    int cube40;              // every streamed robot is 40 x 40 x 40 (compile-time strides)
    // checkpoint of the state at the start of this step (NULL: none), per corner
    float4* ckpt_u;
    float4* ckpt_v;
    // record of this step for the adjoint (NULL: none), per corner: u before the update with the
    // contact mode in .w, and the horizontal spring force before contact
    float4* rec_u;
    float2* rec_f;
};
cudaError_t launch_step_streamed(const StreamArgs& a, int n, int max_corners, cudaStream_t s);

// Streamed adjoint (robots too large for one SM): records, adjoints and the per-spring
// sensitivity sums live in device memory; one launch per reverse step does the spring part of
// step j and the mass part of step j - 1 (which needs only the corner's own adjoints).
struct StreamAdjArgs {
    PopView pv;
    const uint32_t* cflags;
    const float* prm;        // per robot at 39 * moff: [3][13][C]
    const uint8_t* mat;      // kept material per voxel
    const float4* u0;        // any state array: rest height z0 in .w
    const float4* rec_u;     // spring part: record of step j (u before the update, mode in .w)
    const float4* mrec_u;    // mass part: record of step j - 1 (NULL: no mass part)
    const float2* mrec_f;    //            its horizontal spring force before contact
    const float4* lF_in;     // adjoint of the summed spring force at step j (read, neighbours too)
    float4* lF_out;          // the same at step j - 1 (written by the mass part)
    float4* lu;              // adjoint of u (per corner)
    float4* lv;              // adjoint of v
    float* acc;              // per robot at 39 * moff: [3][13][C] sensitivity sums to k, alpha L0, beta L0
    const float2* sc;        // sin / cos of w t of the recorded call
    int step;                // j, index of the spring part's step in the recorded call (-1: none)
    const double* dL_df;
    StepConst c;
    const int* robots;       // streamed robots (grid.y)
    int n_robots;
    int cube40;              // every streamed robot is 40 x 40 x 40 (compile-time strides)
    float* g_k;              // per voxel accumulators
    float* g_a;
    float* g_b;
};
cudaError_t launch_stream_adj_init(const StreamAdjArgs& a, int max_corners, cudaStream_t s);
cudaError_t launch_stream_adj_step(const StreamAdjArgs& a, int max_corners, cudaStream_t s);
cudaError_t launch_stream_adj_voxels(const StreamAdjArgs& a, int max_corners, cudaStream_t s);

// Cluster lattice path (robots cut into q <= 8 slabs of <= 768 corners, one CTA each, slabs
// exchanging boundary positions and forces through distributed shared memory).
struct ClusterArgs {
    PopView pv;
    const uint32_t* cflags;
    const float* prm;        // per robot at 39 * moff: [3][13][C]
    float4* u;               // per corner displacement (rest height in .w)
    float4* v;
    const float2* sc;        // sin / cos of w t per step of this call
    int nsteps;
    StepConst c;
    const int* robots;       // robots of this launch, one cluster each
    int q;                   // CTAs per cluster
};
int cluster_max_threads();
cudaError_t launch_step_cluster(const ClusterArgs& a, int n_robots, size_t smem, cudaStream_t s);

// The paper's organisation (baseline): one launch per robot per pass, two passes per step.
cudaError_t launch_step_plain_robot(const int2* ab, const float4* prm, const int* mass_corner, float4* u,
                                    float4* v, float* F, int S, int M, int nx, int ny, const float2* sc, int n,
                                    StepConst c, cudaStream_t s);

// Adjoint of the lattice stepping over one recorded call (see adjoint.cu).
struct AdjointArgs {
    PopView pv;
    const uint32_t* cflags;
    const float* prm;
    const uint8_t* mat;      // kept material per voxel
    const float4* u0;        // any state array: rest height z0 in .w
    const float4* rec_u;     // this segment's records, [n - n0][rec_stride]: state before the update, mode in .w
    const float2* rec_f;     //   and the horizontal spring force before contact
    int64_t rec_stride;
    int n0, n1;              // steps of the segment within the recorded call
    int first;               // the latest segment: start from the adjoint of the fitness
    int last;                // the earliest segment: scatter the sensitivity sums onto voxels
    float4* lu;              // adjoints of u and v carried between segments (per corner)
    float4* lv;
    float* acc;              // per robot at 39 * moff: [3][13][C] sensitivity sums carried between segments
    const float2* sc;        // sin / cos of w t per step of the recorded call
    StepConst c;
    const double* dL_df;     // [P]
    const int4* items;
    const int* item_robots;
    int n_items;
    int cube8;               // every item is one 8 x 8 x 8 robot in a 768-thread slot
    int* queue;
    float* g_k;              // per voxel: dL/dk_v, dL/d(alpha_v), dL/d(beta_v) accumulators
    float* g_a;
    float* g_b;
};
cudaError_t launch_adjoint_lattice(const AdjointArgs& a, int grid, int threads, size_t smem,
                                   cudaStream_t s);
cudaError_t launch_adjoint_voxels(const uint8_t* mat, const float* w, const float* kappa,
                                  const float* phi, MatConst mc, const float* g_k, const float* g_a,
                                  const float* g_b, int64_t n, float* g_w, float* g_kappa,
                                  float* g_phi, cudaStream_t s);
int lattice_max_threads();
// Shared-memory bandwidth probe: grid blocks of 1024 threads, iters rounds of 8 16-byte loads.
cudaError_t launch_probe_smem(int grid, int iters, float* sink, cudaStream_t s);
size_t probe_smem_bytes_per_iter(int grid);
constexpr int kLatticeSlotVec4 = 15;     // shared float4 per corner slot: u, v, 13 force planes
cudaError_t launch_step_lattice(const LatticeArgs& a, int grid, int threads, size_t smem,
                                cudaStream_t s);
// Mass-packed lattice kernel: 768-thread blocks shared by groups of robots sized by mass count.
cudaError_t launch_step_lattice_packed(const LatticeArgs& a, int grid, size_t smem, cudaStream_t s);
size_t resident_smem_bytes(int max_mass, int max_spring_smem, int accumulate);

cudaError_t launch_fitness(PopView pv, const int* mass_corner, const float4* u, const float4* x0,
                           float dead_bound, double* out, cudaStream_t s);

cudaError_t launch_evo_rank(const double* fitness, int P, int* order, cudaStream_t s);
cudaError_t launch_elite_weights(const int* order, const double* fitness, int P, int E, double* w,
                                 cudaStream_t s);
cudaError_t launch_evo_children(const float* gin, float* gout, const int* order, int P, int G,
                                int E, uint64_t seed, uint64_t gen, uint32_t thresh, float sigma,
                                uint32_t keep, int* parents, uint8_t* mask, cudaStream_t s);

cudaError_t launch_compact_state(PopView pv, const int* mass_corner, const float4* src,
                                 const float4* add, float* dst, const int64_t* dst_off, cudaStream_t s);

// Population diversity totals (see fitness_evo.cu): totals[0] = sum of squared deviations of the
// genomes from their mean, totals[1] = number of (robot pair, voxel) disagreements.
cudaError_t launch_diversity(const float* genomes, int P, int G, const uint8_t* mat, int V, double* totals,
                             cudaStream_t s);

// Record a failure message for sim_last_error() on this thread and return `st`.
sim_status vx_fail(sim_status st, const char* fmt, ...);

}  // namespace vx
