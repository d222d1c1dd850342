/*
 * voxsim.h -- C ABI of the GB300 (sm_103a) voxel soft-robot co-design library.
 *
 * The library runs, on one GPU, the data-parallel hot path of "CUDA-Accelerated Soft Robot
 * Neural Evolution with Large Language Model Supervision" (L. Zhang, arXiv 2405.00698):
 *   decode (Gaussian positional encoding, Eq. (1), and the MLP spatial query, Section II-C)
 *   -> largest connected component -> masses / springs (Section II-A, Table II)
 *   -> batched time stepping (spring and mass updates, Section II-C)
 *   -> centroid fitness -> elite selection, crossover, mutation (Section II-C, Table I)
 *   and the reverse-mode adjoint of the time stepping.
 *
 * Conventions shared by every entry point
 *   - Plain C types only.  A `mem` argument says where a caller buffer lives:
 *     SIM_MEM_HOST (ordinary or pinned host memory) or SIM_MEM_DEVICE (device memory of the
 *     context's GPU, e.g. a torch tensor's data_ptr()).
 *   - The caller owns every buffer it passes.  The library copies what it needs before the call
 *     returns and keeps no caller pointer afterwards.
 *   - Work is enqueued on the context's stream.  Calls that write host memory synchronise that
 *     stream before returning; device-to-device calls are asynchronous.
 *   - Nothing aborts or exits.  Every call returns a sim_status; sim_last_error() gives the
 *     message of the most recent failure on the calling thread.
 *   - One context per thread at a time; a context is not safe for concurrent calls.
 *
 * Material ids (Section II-A): 0 empty, 1 expanding muscle, 2 contracting muscle,
 * 3 soft tissue, 4 bone.
 */
#ifndef VOXSIM_H
#define VOXSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = 1,    /* bad argument (size, pointer, mode, out-of-range value) */
    SIM_ENOMEM = 2,    /* device or host allocation failed */
    SIM_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    SIM_ESTATE = 4,    /* call out of order (e.g. stepping before a population is set) */
    SIM_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    SIM_ENUMERIC = 6   /* non-finite values where finite ones are required */
} sim_status;

enum { SIM_MEM_HOST = 0, SIM_MEM_DEVICE = 1 };

/* How sim_set_population reads `genomes`. */
enum {
    SIM_MODE_MATERIALS = 0, /* uint8 material id per voxel, all robots' grids concatenated */
    SIM_MODE_LOGITS = 1,    /* float32 [voxels][5] material scores; material = argmax (lowest id
                               on ties), material weight 1 */
    SIM_MODE_MLP = 2,       /* float32 [P][20998] MLP genomes, queried at every voxel centre */
    SIM_MODE_PARAMS = 3,    /* const sim_voxel_params*: materials plus per-voxel weight,
                               stiffness and phase (the differentiable parametrisation) */
    SIM_MODE_PARAM_ROWS = 4 /* const sim_param_rows*: the same parametrisation as one genome row
                               per robot, [w | kappa | phi], for the genetic operators */
};

/* Force accumulation of the time stepping kernels. */
enum {
    SIM_ACC_AUTO = 0,   /* library choice (measured default) */
    SIM_ACC_ATOMIC = 1, /* per-spring threads add into per-mass accumulators atomically */
    SIM_ACC_GATHER = 2  /* every mass sums its springs' forces in a fixed order (lattice-gather
                           kernel, a cluster of lattice blocks for robots of up to 8 x 768
                           corners in whole layers, or the streamed path): bit-reproducible */
};

/* Execution path of the time stepping. */
enum {
    SIM_PATH_AUTO = 0,      /* resident for robots whose masses fit on chip, streamed otherwise */
    SIM_PATH_RESIDENT = 1,  /* state in shared memory for all steps of a call: one thread-block
                               group per robot, or a cluster of blocks for a larger robot */
    SIM_PATH_STREAMED = 2,  /* structure-of-arrays state in device memory, one pass per step */
    SIM_PATH_PLAIN = 3      /* the paper's organisation, kept as a baseline: per robot and step one
                               launch with a thread per spring (atomic force sums in device
                               memory) and one with a thread per mass */
};

/* MLP query kernel. */
enum {
    SIM_MLP_TENSOR = 0, /* tcgen05 tensor-core kernel, accumulators in TMEM, operands by TMA */
    SIM_MLP_SIMT = 1    /* CUDA-core kernel with the same bfloat16 rounding points */
};

/* Variant of the lattice-gather kernel (robots of at most 768 corners on the resident path).
 * All give identical bits; they differ in how threads share the work. */
enum {
    SIM_LATTICE_AUTO = 0,   /* library choice (measured default, autotuned): one robot per slot,
                               or the robots in mass-sized groups (SIM_LATTICE_PACKED) once their
                               masses fill less than 55 % of their slots' threads */
    SIM_LATTICE_CORNER = 1, /* a thread per mass evaluates its 13 forward lattice directions, one
                               robot per block slot sized by its grid corners */
    SIM_LATTICE_COMPACT = 2,/* along each direction the existing springs are packed onto the
                               first threads, so warps skip absent springs; each mass then sums
                               its springs' forces from shared memory */
    SIM_LATTICE_PACKED = 3  /* the per-mass scheme of SIM_LATTICE_CORNER with several robots per
                               768-thread block, each in a group of threads sized by its mass
                               count (force rows indexed by the receiving thread), also for
                               robots of more than 768 corners but at most 768 masses; for
                               robots of up to 768 corners measured slower than
                               SIM_LATTICE_CORNER until they fill less than about 55 % of their
                               slots (the default then picks it) */
};

/* Physics constants (Table II; the workload configurations override some of them) and
 * execution choices. */
typedef struct {
    double dt;          /* time step [s] */
    double gravity;     /* [m/s^2] */
    double mass;        /* point mass per voxel corner [kg] */
    double edge;        /* voxel edge = original rest length [m] */
    double damping;     /* velocity multiplier applied every step (1 = none) */
    double k_ground;    /* ground penalty stiffness [N/m] */
    double mu_s;        /* static friction coefficient */
    double mu_k;        /* kinetic friction coefficient */
    double freq;        /* muscle actuation frequency [Hz] */
    double dead_bound;  /* |coordinate| beyond this marks a robot dead [m] */
    double k_mat[5];    /* stiffness per material [N/m] */
    double amp_mat[5];  /* actuation amplitude per material, fraction of the rest length */
    double phase_mat[5];/* actuation phase per material [rad] */
    int32_t ground_on;  /* 0 removes the ground plane */
    int32_t accumulate; /* SIM_ACC_* */
    int32_t path;       /* SIM_PATH_* */
    int32_t threads;    /* threads per robot on the resident path; 0 = autotuned */
    int32_t mlp_kernel; /* SIM_MLP_TENSOR (tcgen05, default) or SIM_MLP_SIMT (CUDA cores) */
    int32_t lattice;    /* SIM_LATTICE_* */
    double spring_zeta; /* spring dashpot damping ratio (Table II: 0.1; 0 in the configurations):
                           c_s ((v_b - v_a) . u) u with c_s = 2 zeta sqrt(k_s mass / 2) */
    double ground_zeta; /* ground damping ratio (Table II: 0.1): -2 zeta sqrt(k_ground mass) v_z
                           below the ground.  The adjoint requires both to be 0 */
} sim_params;

/* Per-voxel parametrisation for SIM_MODE_PARAMS (all arrays cover every voxel of every grid):
 * stiffness k_v = w_v * kappa_v, actuation amplitude a_v = w_v * amp_mat[material], phase phi_v. */
typedef struct {
    const uint8_t* mat;
    const float* w;
    const float* kappa;
    const float* phi;
} sim_voxel_params;

/* SIM_MODE_PARAM_ROWS: every robot on one grid shape of V voxels; row r of `rows` (float32
 * [P][3 V]) holds robot r's per-voxel w (entries 0 .. V-1), kappa (V .. 2V-1) and phi (2V ..
 * 3V-1), voxel order as in sim_set_population; `mat` is uint8 [P][V]. */
typedef struct {
    const uint8_t* mat;
    const float* rows;
} sim_param_rows;

/* Evolution rates (Table I; configuration values: elites 25 %, sigma 0.05, rate 0.1). */
typedef struct {
    int32_t elites;         /* E >= 1: genomes kept unchanged */
    uint32_t mut_threshold; /* a gene mutates when its 32-bit draw is below this
                               (floor(rate * 2^32)) */
    float sigma;            /* standard deviation of the Gaussian mutation */
    uint32_t keep_threshold;/* crossover rate below 1 (Table I: 0.4): a child whose draw
                               (c, crossover) is below floor((1 - rate) 2^32) copies parent A;
                               0 = every child is a crossover */
    uint64_t seed;          /* seed of the counter-based generator */
} evo_params;

typedef struct voxsim_ctx voxsim_ctx;

/* Create a context on CUDA device `device`, enqueueing all work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  `p` is copied.  Errors: SIM_EINVAL for a
 * NULL out pointer or non-positive dt / mass / edge, SIM_ECUDA if the device cannot be used. */
sim_status sim_create(const sim_params* p, int32_t device, void* cuda_stream, voxsim_ctx** out);

/* Release every device buffer of the context (synchronises its stream first) and the context
 * itself, which must not be used afterwards.  NULL is a no-op.  Always returns SIM_OK. */
sim_status sim_destroy(voxsim_ctx* ctx);

/* Message of the most recent failed call on this thread ("" if none).  Valid until the next
 * call on this thread.  ctx may be NULL (the message is per thread, not per context). */
const char* sim_last_error(const voxsim_ctx* ctx);

/* The device status words that sim_set_population's kernels raise, mapped to the status and
 * message the call returns: words[1] bit 2 (a bounded wait of the tensor-core MLP query gave up;
 * the kernel drains its copies and MMAs before it frees its tensor memory) and words[0] bit 0 (the
 * component labelling hit its iteration bound) give SIM_ETIMEOUT, words[0] bit 1 (a material
 * id out of range in device-memory genomes) SIM_EINVAL, none SIM_OK.  words[2] bit 3 is the
 * stepping's (a segment of the lattice step gave up its bounded wait for its robots' previous
 * segment, see sim_step_n), reported as SIM_ETIMEOUT by sim_fitness into host memory.
 * words: host int32 [4].
 * Needs no device: it lets a caller (and the test-suite) check the mapping without making a
 * device-side wait run out.  The paper has no counterpart.  Errors: SIM_EINVAL for NULL. */
sim_status sim_check_status_words(const int32_t* words);

/* Replace the population: P robots, robot r on a dims[3r] x dims[3r+1] x dims[3r+2] voxel grid
 * (each 1..64; host array).  Voxel (i, j, k) of robot r is entry i + nx*(j + ny*k) of its grid,
 * grids concatenated in robot order.  Decoding by `mode` (see SIM_MODE_*); for SIM_MODE_MLP
 * `B` is the float32 [128][3] Gaussian encoding matrix of Eq. (1) in the same memory as
 * `genomes` and all robots must share one grid shape.  Then, per robot: only the largest
 * face-connected component of occupied voxels is kept (size ties keep the component holding
 * the smallest voxel index); masses sit at the corners of kept voxels (ascending corner id
 * ci + (nx+1)*(cj + (ny+1)*ck)); springs join the 28 corner pairs of every kept voxel, one
 * spring per distinct pair, with stiffness and actuation terms averaged over the kept voxels
 * that share it; the initial pose is the lattice at rest with its lowest mass at z = 0, and the
 * step counter restarts at 0.  Errors: SIM_EINVAL (sizes, mode, pointers, material ids out
 * of range), SIM_ENOMEM, SIM_ETIMEOUT (a bounded device-side wait or iteration of the decode or
 * topology kernels gave up, see sim_check_status_words). */
sim_status sim_set_population(voxsim_ctx* ctx, int32_t P, const int32_t* dims, int32_t mode,
                              const void* genomes, const float* B, int32_t mem);

/* Advance every robot by n_steps time steps (Section II-C: each spring's force with its
 * sinusoidal rest-length actuation, accumulation onto masses, gravity, ground contact with
 * static / kinetic friction, semi-implicit Euler with velocity damping; Table II).  Time of
 * step n is n * dt from the last sim_set_population.  Kinetic friction removes mu_k F_n along
 * the horizontal force but never more than that force (with Table II's mu_s < mu_k it would
 * otherwise reverse it).  When checkpointing is on
 * (sim_set_checkpointing), the call records the states the adjoint needs.  With more lattice
 * work items than SMs (and at least 512 steps) the resident lattice step runs every item's steps
 * as segments from one queue, each segment waiting (bounded, on the device) for its robots'
 * previous one; the results are the same bits as whole runs.  A wait that gives up is reported
 * by the next sim_fitness into host memory (SIM_ETIMEOUT).
 * Errors: SIM_ESTATE without a population, SIM_EINVAL for n_steps < 0. */
sim_status sim_step_n(voxsim_ctx* ctx, int32_t n_steps);

/* Fitness of every robot: centroid displacement along +x since the initial pose (the paper
 * names "fitness", Section III; the displacement is the workloads' definition), reduced in
 * FP64.  Empty robots score 0; a robot with a non-finite coordinate, or one beyond dead_bound,
 * scores -infinity.  out: double [P] in `mem` (host: the call synchronises the stream).
 * Errors: SIM_ESTATE without a population, SIM_EINVAL for a NULL out or a `mem` other than
 * SIM_MEM_HOST / SIM_MEM_DEVICE, SIM_ECUDA; into host memory also SIM_ETIMEOUT when a segmented
 * lattice step since the population was set gave up a wait (its robots' state is invalid;
 * the fitness is still written). */
sim_status sim_fitness(voxsim_ctx* ctx, double* out, int32_t mem);

/* One generation of the evolutionary step, fully on the GPU (Section II-C; Table I):
 * rank by fitness (descending, ties by ascending index, NaN as -infinity); copy the E best
 * genomes unchanged into rows 0..E-1 in rank order; every row c >= E is a uniform crossover of
 * two elites (parent ranks floor(u E / 2^32) from the draws (c, parent A / B); gene j from
 * parent A when the top bit of draw (c, j, mask) is set) followed by Gaussian mutation
 * (when draw (c, j, mutate) < mut_threshold add sigma * sqrt(-2 ln u1) cos(2 pi u2),
 * u1 = (draw(c, j, u1) + 1) / 2^32, u2 = draw(c, j, u2) / 2^32).  A draw is the high 32 bits of
 * SplitMix64 output number ((((generation << 16 | c) << 26 | j) << 3) | purpose) of the stream
 * seeded with e->seed; purposes: parent A 0, parent B 1, mask 2, mutate 3, u1 4, u2 5,
 * crossover 6 (drawn at gene 0; only with a keep_threshold).
 * fitness: double [P]; genomes_in / genomes_out: float [P][G] (may alias: the input is copied
 * first); parents_out: int32 [P][2] or NULL (elites name themselves twice); mask_out: uint8
 * [P][G] or NULL (1 = gene from parent A, 0 for elites).  All device memory of the context's
 * GPU.  genomes_in may be NULL when the last sim_set_population read its genome rows (MLP
 * genomes, material logits or parameter rows) from host memory: the library's device copy of
 * them is then the input, so a population that starts on the host is uploaded once.
 * Limits: 1 <= E <= P <= 65536, G <= 2^26, generation < 2^19.
 * Errors: SIM_EINVAL, SIM_ENOMEM (library scratch), SIM_ESTATE (NULL genomes_in without host
 * genome rows; P x G must then equal their size). */
sim_status evo_generation(voxsim_ctx* ctx, const double* fitness, const float* genomes_in,
                          float* genomes_out, int32_t P, int32_t G, const evo_params* e,
                          uint64_t generation, int32_t* parents_out, uint8_t* mask_out);

/* evo_generation without any device allocation, for callers that cannot call cudaMalloc: a
 * serving or control process whose memory pool already holds the whole device (another
 * cudaMalloc would fail), or code that must not allocate once its loop is running (cudaMalloc
 * and cudaFree can synchronise the device and stall the loop).  The paper has no counterpart; it
 * is the same operation as evo_generation (same kernels, same results bit for bit) with two
 * differences:
 *   - it needs no context: the caller passes the CUDA stream (NULL = legacy default stream) and
 *     the work runs on the current device;
 *   - its only scratch (the rank order of the population) is a fixed device array of 16384
 *     entries (64 KB) built into the library, which every GPU that loads the library keeps until
 *     the process exits.  P above 16384 is rejected with SIM_EINVAL, and so are overlapping
 *     genomes_in / genomes_out (there is no room for a copy).
 * Every call on a device shares that array and leaves its contents behind (each call overwrites
 * all the entries it reads, so nothing needs clearing); calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress with that device
 * current) and keeps it for the life of the process; make that first call before any stream
 * capture.  The kept address does not survive cudaDeviceReset (the array may come back at
 * another address): a process that resets a device must not call this entry point on that
 * device afterwards.  Errors as for evo_generation. */
sim_status evo_generation_static(const double* fitness, const float* genomes_in,
                                 float* genomes_out, int32_t P, int32_t G, const evo_params* e,
                                 uint64_t generation, int32_t* parents_out, uint8_t* mask_out,
                                 void* cuda_stream);

/* Lamarckian gradient step of the gradient-assisted co-design variant (project extension: the
 * paper evolves with genetic operators only; this keeps them unchanged and moves chosen genomes
 * uphill along the adjoint's gradient before they breed).  Genomes are SIM_MODE_PARAM_ROWS rows
 * (float32 device [P][G], G = 3 V) of the context's current population (P robots on one grid of
 * V voxels); g_w, g_kappa, g_phi are sim_backward's outputs for that population (device, one
 * entry per voxel).  For every robot r in rows (host int32 [n_rows], each in 0 .. P-1; NULL =
 * every robot) and gene j with gradient d_rj (g_w, g_kappa or g_phi of voxel j mod V) and step
 * eta_j (eta_w, eta_kappa or eta_phi, one per segment since the three scale differently):
 *     genome_rj <- min(max(fmaf(eta_j, d_rj, genome_rj), lo_j), hi_j)
 * lo, hi: device float32 [G] bounds, or NULL for none.  Enqueued on the context's stream.
 * Errors: SIM_ESTATE without a population, SIM_EINVAL (sizes, null pointers, a row out of range,
 * a population that is not on one grid shape). */
sim_status evo_gradient_step(voxsim_ctx* ctx, float* genomes, int32_t P, int32_t G, const float* g_w,
                             const float* g_kappa, const float* g_phi, const int32_t* rows,
                             int32_t n_rows, float eta_w, float eta_kappa, float eta_phi,
                             const float* lo, const float* hi);

/* The elites of a generation as adjoint weights, on the GPU (gradient-assisted variant, project
 * extension): robots are ranked as evo_generation ranks them (fitness descending, ties by
 * ascending index, NaN as -infinity) and weights[r] = 1 for the E best robots whose fitness is
 * finite, 0 for every other robot.  Passed to sim_backward as dL_df it gives the gradient of the
 * elites' summed fitness; no host round trip is needed to pick them.  fitness, weights: double
 * [P], device memory; enqueued on the context's stream.  Errors: SIM_EINVAL (null pointers, P
 * outside 1..65535, E outside 0..P), SIM_ENOMEM. */
sim_status evo_elite_weights(voxsim_ctx* ctx, const double* fitness, int32_t P, int32_t E, double* weights);

/* Turn state checkpointing on (every k_steps steps, k_steps >= 1) or off (0).  While on, each
 * sim_step_n call records the state at its start and every k_steps steps after, which
 * sim_backward replays (device memory: two float4 per grid corner per checkpoint, plus during
 * sim_backward k_steps records of 24 bytes per corner).  Every robot must run on a deterministic
 * kernel: while checkpointing is on, robots that would run on the atomic resident kernel run on
 * the streamed path instead (the population's plan is rebuilt when the setting changes).
 * The paper preset's dashpots (spring_zeta, ground_zeta != 0) are not differentiated.
 * Errors: SIM_EINVAL (k_steps < 0, SIM_ACC_ATOMIC, damped parameters), SIM_ENOMEM. */
sim_status sim_set_checkpointing(voxsim_ctx* ctx, int32_t k_steps);

/* Keep every step's record of the recorded run (on = 1) instead of only its checkpoints
 * (on = 0, the default).  While on and checkpointing is on (sim_set_checkpointing), each
 * sim_step_n call also stores, for every step and every grid corner, the state before the update
 * with its contact mode and the horizontal spring force before contact (24 bytes per corner per
 * step: n_steps x 24 B x the population's grid corners, e.g. about 18 GB for 512 robots of
 * 8x8x8 voxels over 2000 steps), and sim_backward sweeps those records backwards in one pass
 * without replaying the forward steps (the same forward run and contact modes bit for bit, the
 * same gradients up to the order of the per-voxel atomic sums), for the robots on the resident
 * lattice kernel and on the streamed path alike.  Records written under another routing of robots
 * to kernels than the current one (a sim_autotune in between) are not used: the checkpoints are
 * replayed instead.  A sim_step_n call that cannot allocate the records fails with SIM_ENOMEM.
 * Changing the setting discards the recorded run; turning it off frees the records.
 * Errors: SIM_EINVAL (on not 0 or 1). */
sim_status sim_set_trajectory_records(voxsim_ctx* ctx, int32_t on);

/* Reverse-mode gradient of L = sum_r dL_df[r] * fitness_r over the most recent recorded
 * sim_step_n call, with respect to the per-voxel material weight w, stiffness kappa and
 * actuation phase phi (k_v = w_v kappa_v, a_v = w_v amp_mat[material], phase phi_v).  The
 * forward steps are recomputed from the checkpoints segment by segment, bit-identically, and
 * each segment is swept backwards; contact modes of the forward run are held fixed.  Robots on
 * the resident lattice kernels and robots on the streamed path are both differentiated (each
 * by its own sweep).  The checkpoints are left intact, so the call may be repeated with another
 * dL_df on the same recorded run.  Empty voxels get 0.  dL_df: double [P]; g_w, g_kappa,
 * g_phi: float, one entry per voxel of every grid (concatenated as in sim_set_population); all
 * device memory.  The resident robots' segment replays run on a second stream that the context
 * creates on first use, ordered against the context's stream by events (the call's work starts
 * after, and ends before, what the context's stream holds around it).
 * Errors: SIM_ESTATE without a recorded run, SIM_EINVAL, SIM_ENOMEM. */
sim_status sim_backward(voxsim_ctx* ctx, const double* dL_df, float* g_w, float* g_kappa,
                        float* g_phi);

/* Contact mode of every corner of robot `robot` at every step of the most recent recorded
 * sim_step_n call (checkpointing on): out[n * C + c] for step n and grid corner c of the robot's
 * C corners, 0 = free (or no mass at that corner), 1 = stuck, 2 = slipping, 3 = slipping with
 * the kinetic friction saturated (mu_k F_n >= |F_h|, possible only when mu_k > mu_s as in
 * Table II: the horizontal force is cancelled, never reversed) (Section II-C, Table II: ground
 * contact with static and kinetic friction).  The checkpoint segments are
 * replayed bit-identically to read them.  out: host uint8 [n_steps][C].  Synchronises the
 * stream.  Errors: SIM_ESTATE without a recorded run, SIM_EINVAL. */
sim_status sim_get_contact_modes(voxsim_ctx* ctx, int32_t robot, uint8_t* out);

/* Impose the contact modes of robot `robot` on the steps that follow sim_set_population
 * (analysis and testing: differentiating the step map along another run's contact decisions,
 * such as those of an FP64 reference run, so that both sides follow the same piecewise-smooth
 * map).  modes: host uint8 [n_steps][C] over the robot's C grid corners in the layout of
 * sim_get_contact_modes (0 free, 1 stuck, 2 slipping, 3 saturated slip; corners without a mass
 * are ignored).  At run step n < n_steps (counted from sim_set_population) every mass of the
 * robot takes modes[n][corner] instead of deciding it from its state: free adds no ground force;
 * the three contact modes add F_n = k_ground (-z) whatever the sign of z, then zero the
 * horizontal force and velocity (stuck), remove mu_k F_n along F_h (slipping) or zero the
 * horizontal force (saturated).  Later steps decide freely.  Every imposed robot covers the same
 * n_steps; NULL modes clears every imposition; sim_set_population clears them too.  While modes
 * are imposed, every robot of at most 768 corners steps on the per-corner lattice kernel, also in
 * the replays of sim_backward and sim_get_contact_modes, which therefore follow the same modes.
 * Errors: SIM_ESTATE without a population, SIM_EINVAL (robot out of range or larger than a
 * lattice block, a mode above 3, another n_steps than the robots already imposed, damped
 * physics, the streamed, plain or atomic organisation), SIM_ENOMEM. */
sim_status sim_impose_contact_modes(voxsim_ctx* ctx, int32_t robot, const uint8_t* modes, int32_t n_steps);

/* Population diversity (Fig. 3(b) plots a "diversity curve" without defining it; these are the
 * definitions used here), FP64 on the GPU:
 *   out[0] genome diversity: root mean square of the pairwise Euclidean distances between the P
 *          genomes (device float [P][G]; NULL skips it and leaves NaN);
 *   out[1] morphology diversity: mean over robot pairs of the fraction of voxels whose kept
 *          materials differ, for the current population when it has P robots on one grid shape
 *          (NaN otherwise).
 * out: host double [2].  Synchronises the stream.  Errors: SIM_EINVAL for P < 2. */
sim_status sim_diversity(voxsim_ctx* ctx, const float* genomes, int32_t P, int32_t G, double* out);

/* Per-size autotuner of the stepping kernels (project-written; the paper has no counterpart).
 * Robots are grouped by grid-corner count into 10 classes (up to 64, 128, 192, 256, 384, 768,
 * 1536, 2560, 5120 corners, and more).  For every class present in the population, each
 * admissible kernel (the lattice-gather kernel in its two variants, the cluster lattice kernel,
 * the atomic resident kernel at three block sizes, the lattice kernel in mass-sized thread groups
 * for sparse robots of more than 768 corners, the streamed path) is timed on up to six robots
 * per SM of that class for n_steps steps from
 * the current state (CUDA events), and the fastest is kept for that class.  The state is
 * restored afterwards; the choices persist for later populations of this context.  The trial
 * runs record nothing: a recorded run (sim_step_n with checkpointing on) stays available to
 * sim_backward, which replays its checkpoints.  Modes that
 * require bit-reproducibility (SIM_ACC_GATHER, checkpointing) only consider deterministic
 * kernels.  kind_out / threads_out: int32 [10] host arrays (either may be NULL) receiving per
 * class 0 = lattice (per corner), 1 = atomic resident, 2 = streamed, 3 = lattice
 * (direction-compacted), 4 = cluster of lattice blocks (robots cut into slabs of whole corner
 * layers, one block each), 5 = lattice in thread groups sized by mass count (robots of more than
 * 768 corners but at most 768 masses; larger ones of the class take the atomic kernel, or the
 * cluster when bit-reproducibility is required), and the atomic kernel's block size.
 * Synchronises the stream.  Errors: SIM_ESTATE without a population, SIM_EINVAL. */
sim_status sim_autotune(voxsim_ctx* ctx, int32_t n_steps, int32_t* kind_out, int32_t* threads_out);

/* Mass and spring count of every robot (host arrays of P int32; either may be NULL).
 * Synchronises the stream.  Errors: SIM_ESTATE without a population. */
sim_status sim_get_counts(voxsim_ctx* ctx, int32_t* n_masses, int32_t* n_springs);

/* Current state: positions and velocities (float32 [total masses][3], robots in order, masses
 * in ascending corner order); mass_offsets: int32 [P+1] prefix offsets (host) or NULL.  Any
 * output may be NULL.  mem applies to x_out and v_out.  Synchronises the stream.
 * Errors: SIM_ESTATE without a population, SIM_EINVAL for an unknown `mem`, SIM_ENOMEM,
 * SIM_ECUDA. */
sim_status sim_get_state(voxsim_ctx* ctx, float* x_out, float* v_out, int32_t* mass_offsets,
                         int32_t mem);

/* Decoded voxels before / after the largest-component filter and the per-voxel parameters
 * actually simulated (host arrays over all voxels; any may be NULL).  Synchronises the stream.
 * Errors: SIM_ESTATE without a population, SIM_ECUDA. */
sim_status sim_get_voxels(voxsim_ctx* ctx, uint8_t* mat_decoded, uint8_t* mat_kept, float* w,
                          float* kappa, float* phi);

/* Topology (host arrays, robots concatenated, sized by sim_get_counts): mass_corner int32 per
 * mass; spring_ab int32 [springs][2] (mass indices within the robot, a < b, sorted by (a, b));
 * spring_params float [springs][4] = rest length, stiffness, alpha, beta with the actuated rest
 * length L0 (1 + alpha sin(w t) + beta cos(w t)).  Any may be NULL.  Synchronises the stream.
 * Errors: SIM_ESTATE without a population, SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_get_topology(voxsim_ctx* ctx, int32_t* mass_corner, int32_t* spring_ab,
                            float* spring_params);

/* Since the last call: cumulative device time of the time-stepping kernels (milliseconds,
 * CUDA events on the context's stream) and the number of kernels the library launched (all
 * entry points).  Synchronises the stream and resets both.  Either output may be NULL.
 * Errors: SIM_EINVAL for a NULL context, SIM_ECUDA. */
sim_status sim_get_timing(voxsim_ctx* ctx, double* step_ms, int64_t* launches);

/* Measured shared-memory bandwidth of the context's device (GB/s, all SMs): two 1024-thread
 * blocks per SM stream conflict-free 16-byte loads from their shared memory for about 5 ms
 * (after a warm-up launch), timed with CUDA events on the context's stream.  The resident
 * stepping kernels keep their state in shared memory, so this, not HBM, is the roofline they
 * are measured against.  Synchronises the stream; allocates and frees a scratch array of 8 B
 * per SM.  Errors: SIM_EINVAL for a NULL context or output, SIM_ECUDA. */
sim_status sim_measure_smem_bandwidth(voxsim_ctx* ctx, double* gbs);

#ifdef __cplusplus
}
#endif

#endif /* VOXSIM_H */
