// Host side of the C ABI declared in include/voxsim.h: context, device buffers, launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

using namespace vx;

namespace {

thread_local std::string g_err;

sim_status fail(sim_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

}  // namespace

sim_status vx::vx_fail(sim_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

namespace {

sim_status cuda_fail(cudaError_t e, const char* what)
{
    // the error is returned to the caller, so it must not also stay pending in the runtime's
    // last-error state, where the caller's next unrelated CUDA check would find it (a failed
    // allocation leaves the context usable)
    (void)cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define VX_CK(call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);           \
    } while (0)

// A kernel launch through one of the launch_* helpers, counted for sim_get_timing.
#define VX_LAUNCH(ctx, call)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);           \
        (ctx)->launches += 1;                                         \
    } while (0)

// Device buffer that only grows.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t want)
    {
        if (want <= n && p) return cudaSuccess;
        release();
        if (want == 0) want = 1;
        cudaError_t e = cudaMalloc((void**)&p, want * sizeof(T));
        if (e != cudaSuccess) { p = nullptr; n = 0; return e; }
        n = want;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
};

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int64_t full_springs(int nx, int ny, int nz)
{
    const int64_t X = nx, Y = ny, Z = nz;
    const int64_t edges = X * (Y + 1) * (Z + 1) + Y * (X + 1) * (Z + 1) + Z * (X + 1) * (Y + 1);
    const int64_t faces = 2 * (X * Y * (Z + 1) + X * Z * (Y + 1) + Y * Z * (X + 1));
    return edges + faces + 4 * X * Y * Z;
}

}  // namespace

// Size classes by grid-corner count: the six lattice slot sizes, then larger bands.
constexpr int kNumClasses = 10;
constexpr int kClassCorners[kNumClasses] = {64, 128, 192, 256, 384, 768, 1536, 2560, 5120, 1 << 30};
enum { kKindLattice = 0, kKindAtomic = 1, kKindStreamed = 2, kKindLatticeCompact = 3, kKindCluster = 4,
       kKindMassGroups = 5 };

static int class_of(int corners)
{
    for (int k = 0; k < kNumClasses; ++k)
        if (corners <= kClassCorners[k]) return k;
    return kNumClasses - 1;
}

struct voxsim_ctx {
    sim_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;
    // population layout (host copies)
    int P = 0;
    bool have_pop = false;
    std::vector<int> dims;
    std::vector<int64_t> voff, moff, soff;
    std::vector<int> mass_count;   // masses and springs per robot of the current population (host copies)
    std::vector<int> spring_count;
    int64_t V_tot = 0, M_cap = 0, S_cap = 0;
    int max_corner = 0;
    int64_t max_spring_cap = 0;
    int64_t step = 0;
    // lattice work items (robots up to lattice_max_threads() corners), robots on the atomic
    // resident kernel (larger, state still fits one SM) and streamed robots (the rest)
    // (lattice items: the per-corner variant's first, n_items_corner of them, then the
    // direction-compacted variant's)
    int n_items = 0, n_items_corner = 0, n_big = 0, max_big_corner = 0;
    bool has_split = false;        // some lattice items are split (two threads per corner)
    // mass-packed plan of the per-corner lattice robots (SIM_LATTICE_PACKED; used for stepping
    // that records nothing per step; the adjoint's replays run the per-corner plan, same bits)
    int n_pitems = 0;
    bool pitems_cover_corner = false;   // the per-corner robots are in the packed plan too
    size_t pitem_smem = 0;
    DevBuf<int4> d_pitems, d_pgroups;
    // imposed contact modes (sim_impose_contact_modes): per robot the offset of its table in
    // imp_table (-1: none), tables of imp_n steps x the robot's corners; device copies
    bool imp_active = false;
    int imp_n = 0;
    std::vector<int64_t> imp_off;
    std::vector<uint8_t> imp_table;
    DevBuf<uint8_t> d_imp_modes;
    DevBuf<int64_t> d_imp_off;
    void imposed_args(LatticeArgs& a, int64_t step0) const
    {
        if (!imp_active) return;
        a.imp_modes = d_imp_modes.p;
        a.imp_off = d_imp_off.p;
        a.imp_n = imp_n;
        a.imp_step0 = step0;
    }
    bool have_pack = false;   // the packed spring list exists for the current population
    int64_t max_big_spring_cap = 0;
    // per size class (by corner count): kind (0 lattice per corner, 1 atomic, 2 streamed,
    // 3 lattice direction-compacted) and threads per
    // robot of the atomic kernel (0 = from the robot size); set by sim_autotune
    int class_kind[kNumClasses];
    int class_threads[kNumClasses];
    bool tuned = false;
    // atomic-kernel groups (one persistent launch each): robots of one thread count
    struct AtomicGroup { int threads; int first; int count; int max_corner; int64_t max_spring_cap; };
    std::vector<AtomicGroup> atomic_groups;
    // cluster lattice groups (one launch each): robots cut into q slabs
    struct ClusterGroup { int q; int first; int count; };
    std::vector<ClusterGroup> cluster_groups;
    int n_cluster = 0;
    DevBuf<int> d_cluster;
    int n_stream = 0, max_stream_corner = 0;
    bool stream_cube40 = false;  // every streamed robot is 40 x 40 x 40
    bool corner_cube8 = false;   // every per-corner lattice item is one 8 x 8 x 8 robot (768 threads)
    std::vector<int> stream_robots;
    DevBuf<int> d_stream;
    // CUDA graph of the streamed N-step loop, cached by step count (captured on a private
    // non-blocking stream, replayed on the context's stream)
    cudaStream_t capture_stream = nullptr;
    // the resident adjoint's replays run on their own stream (backward_lattice); events: replay
    // of record buffer 0 / 1 done, sweep of record buffer 0 / 1 done, start of the backward
    cudaStream_t replay_stream = nullptr;
    cudaEvent_t ev_bwd[5] = {};
    cudaGraphExec_t stream_graph = nullptr;
    int stream_graph_n = -1;
    const void* stream_graph_key = nullptr;   // buffers the graph was captured with
    const void* stream_graph_ckpt = nullptr;  // checkpoint buffer it writes (NULL: none)
    const void* stream_graph_rec = nullptr;   // whole-trajectory record buffer it writes (NULL: none)
    int stream_graph_every = 0;
    void drop_graph()
    {
        if (stream_graph) cudaGraphExecDestroy(stream_graph);
        stream_graph = nullptr;
        stream_graph_n = -1;
        stream_graph_key = nullptr;
        stream_graph_ckpt = nullptr;
        stream_graph_rec = nullptr;
        stream_graph_every = 0;
    }
    // device buffers
    DevBuf<int> d_dims;
    DevBuf<int64_t> d_voff, d_moff, d_soff, d_tmp_off;
    DevBuf<int> d_nm, d_ns, d_lpt, d_queue, d_status, d_item_robots, d_big, d_grad_rows;
    DevBuf<int> d_progress;      // per lattice item: segments done (segmented queue)
    DevBuf<int4> d_items;
    DevBuf<uint32_t> d_cflags;
    DevBuf<float> d_prm;
    DevBuf<uint8_t> d_in_u8, d_mat_raw, d_mat;
    DevBuf<float> d_in_f32, d_in_f32b, d_in_f32c, d_w, d_kappa, d_phi;
    // floats of genome rows (MLP genomes, material logits or parameter rows) that the last
    // sim_set_population copied from host memory into d_in_f32 (0: none), which evo_generation
    // can take as its input instead of a second upload
    int64_t host_genome_floats = 0;
    DevBuf<int> d_label, d_count, d_corner_mass, d_mass_corner;
    DevBuf<int2> d_sab;
    DevBuf<float4> d_sp, d_spack, d_x0, d_x, d_v, d_x_alt, d_v_alt;
    DevBuf<float> d_plain_f;       // force accumulators of the plain path (3 per corner)
    DevBuf<double> d_x0c, d_keys, d_fit;
    DevBuf<float2> d_sc;
    DevBuf<unsigned char> d_pe;
    DevBuf<float> d_compact;
    // evolution scratch
    DevBuf<int> d_order;
    DevBuf<float> d_gcopy;
    // checkpointing and the adjoint
    int ckpt_every = 0;          // K (0 = off)
    bool rec_valid = false;      // a recorded call is available
    int64_t rec_step0 = 0;
    int rec_n = 0;
    DevBuf<float4> d_ckpt_u, d_ckpt_v;
    DevBuf<float2> d_sc_rec;
    // whole-trajectory records of the lattice-kernel robots (sim_set_trajectory_records): the
    // forward keeps every step's record and sim_backward sweeps them without replaying
    bool keep_records = false;   // requested
    bool rec_full = false;       // the recorded call kept them
    // the routing of robots to kernels changes with every build_work_items; records kept under
    // another routing than the current one are not used (the checkpoints are replayed instead)
    uint64_t items_version = 0, rec_items_version = 0;
    bool records_usable() const { return rec_full && rec_items_version == items_version; }
    DevBuf<float4> d_trec_u;
    DevBuf<float2> d_trec_f;
    // streamed adjoint: per-step records of a segment, adjoints, sensitivity sums, replay state
    DevBuf<float4> d_srec_u, d_slu, d_slv, d_slF0, d_slF1, d_rep_u0, d_rep_u1, d_rep_v0, d_rep_v1;
    DevBuf<float2> d_srec_f;
    DevBuf<float> d_sacc;
    DevBuf<float> d_gk, d_ga, d_gb;
    // timing: one event pair per stepping call since the last sim_get_timing
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double step_ms = 0.0;
    int64_t launches = 0;

    PopView view()
    {
        PopView v;
        v.P = P;
        v.dims = d_dims.p;
        v.voff = d_voff.p;
        v.moff = d_moff.p;
        v.soff = d_soff.p;
        v.n_mass = d_nm.p;
        v.n_spring = d_ns.p;
        return v;
    }
    MatConst matconst() const
    {
        MatConst m;
        for (int i = 0; i < kNumMat; ++i) {
            m.k[i] = (float)p.k_mat[i];
            m.amp[i] = (float)p.amp_mat[i];
            m.phase[i] = (float)p.phase_mat[i];
        }
        return m;
    }
    StepConst stepconst() const
    {
        StepConst c;
        c.dt = (float)p.dt;
        c.dt_over_m = (float)(p.dt / p.mass);
        c.weight = (float)(p.mass * p.gravity);
        c.damping = (float)p.damping;
        c.dt_lo = (float)(p.dt - (double)c.dt);
        c.dtm_lo = (float)(p.dt / p.mass - (double)c.dt_over_m);
        c.weight_lo = (float)(p.mass * p.gravity - (double)c.weight);
        c.damping_c = (float)(1.0 - p.damping);
        c.mu_k_lo = (float)(p.mu_k - (double)(float)p.mu_k);
        c.k_ground = (float)p.k_ground;
        c.mu_s = (float)p.mu_s;
        c.mu_k = (float)p.mu_k;
        c.edge = (float)p.edge;
        c.edge_sqrt2 = (float)(p.edge * 1.4142135623730951);
        c.edge_sqrt3 = (float)(p.edge * 1.7320508075688772);
        c.edge_sq = (float)(p.edge * p.edge);
        c.edge_sq2 = (float)(2.0 * p.edge * p.edge);
        c.edge_sq3 = (float)(3.0 * p.edge * p.edge);
        c.ground_on = p.ground_on ? 1 : 0;
        c.spring_c = (float)(2.0 * p.spring_zeta * std::sqrt(p.mass / 2.0));
        c.ground_c = (float)(2.0 * p.ground_zeta * std::sqrt(p.k_ground * p.mass));
        c.damped = p.spring_zeta > 0.0 ? 1 : 0;
        return c;
    }
};

extern "C" {
static sim_status build_work_items(voxsim_ctx* ctx, const std::vector<int>* subset = nullptr);
static sim_status build_packed_items(voxsim_ctx* ctx, const std::vector<std::vector<std::pair<int, int>>>& lattice,
                                     const std::vector<int>& mass_groups, bool damped);
}

namespace {

sim_status check_ctx(voxsim_ctx* ctx)
{
    if (!ctx) return fail(SIM_EINVAL, "null context");
    return SIM_OK;
}

sim_status copy_in(const void* src, size_t bytes, int mem, void* dst, cudaStream_t s)
{
    if (bytes == 0) return SIM_OK;
    if (!src) return fail(SIM_EINVAL, "null input pointer");
    VX_CK(cudaMemcpyAsync(dst, src, bytes,
                          mem == SIM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    return SIM_OK;
}

sim_status copy_out(void* dst, const void* src, size_t bytes, int mem, cudaStream_t s)
{
    if (bytes == 0) return SIM_OK;
    VX_CK(cudaMemcpyAsync(dst, src, bytes,
                          mem == SIM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (mem == SIM_MEM_HOST) VX_CK(cudaStreamSynchronize(s));
    return SIM_OK;
}

// Status words the decode and topology kernels raise (device int32 [4], zeroed per population):
//   word 0 bit 0: the component labelling of a robot hit its iteration bound;
//   word 0 bit 1: a material id of device-memory genomes was out of range (decoded as empty);
//   word 1 bit 2: a bounded wait of the tensor-core MLP query gave up (the CTA aborted);
//   word 2 bit 3: a segment of the per-corner lattice step gave up waiting for its robots'
//   previous segment (read by sim_fitness into host memory).
sim_status status_from_words(const int32_t* w)
{
    if (w[2] & 8)
        return fail(SIM_ETIMEOUT, "lattice step: a segment's bounded wait on its robots' previous segment "
                                  "gave up (their state is invalid)");
    if (w[1] & 4)
        return fail(SIM_ETIMEOUT, "MLP query: a bounded wait on the tensor-core pipeline gave up "
                                  "(copies and MMAs drained, decoded materials invalid)");
    if (w[0] & 1)
        return fail(SIM_ETIMEOUT, "topology: the component labelling hit its iteration bound");
    if (w[0] & 2) return fail(SIM_EINVAL, "material id out of range 0..4 in device genomes");
    return SIM_OK;
}

__global__ void k_spring_keys(const int* ns, int P, double* keys)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) keys[i] = (double)ns[i];
}

}  // namespace

extern "C" {

const char* sim_last_error(const voxsim_ctx*) { return g_err.c_str(); }

sim_status sim_check_status_words(const int32_t* words)
{
    if (!words) return fail(SIM_EINVAL, "null status words");
    return status_from_words(words);
}

sim_status sim_create(const sim_params* p, int32_t device, void* cuda_stream, voxsim_ctx** out)
{
    if (!p || !out) return fail(SIM_EINVAL, "null argument");
    *out = nullptr;
    if (!(p->dt > 0) || !(p->mass > 0) || !(p->edge > 0))
        return fail(SIM_EINVAL, "dt, mass and edge must be positive");
    if (p->lattice < SIM_LATTICE_AUTO || p->lattice > SIM_LATTICE_PACKED)
        return fail(SIM_EINVAL, "unknown lattice variant %d", p->lattice);
    int ndev = 0;
    VX_CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SIM_EINVAL, "device %d out of range", device);
    DeviceGuard g(device);
    if (!g.ok) return fail(SIM_ECUDA, "cannot select device %d", device);
    voxsim_ctx* c = new (std::nothrow) voxsim_ctx();
    if (!c) return fail(SIM_ENOMEM, "host allocation");
    c->p = *p;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDeviceProperties"); }
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    *out = c;
    return SIM_OK;
}

sim_status sim_destroy(voxsim_ctx* ctx)
{
    if (!ctx) return SIM_OK;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    ctx->drop_graph();
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->replay_stream) {
        cudaStreamSynchronize(ctx->replay_stream);
        cudaStreamDestroy(ctx->replay_stream);
    }
    for (cudaEvent_t e : ctx->ev_bwd)
        if (e) cudaEventDestroy(e);
    delete ctx;   // device buffers are released by their destructors
    return SIM_OK;
}

sim_status sim_set_population(voxsim_ctx* ctx, int32_t P, const int32_t* dims, int32_t mode,
                              const void* genomes, const float* B, int32_t mem)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (P < 0) return fail(SIM_EINVAL, "P must be >= 0");
    if (P > 0 && !dims) return fail(SIM_EINVAL, "null dims");
    if (mem != SIM_MEM_HOST && mem != SIM_MEM_DEVICE) return fail(SIM_EINVAL, "bad mem %d", mem);
    if (mode < SIM_MODE_MATERIALS || mode > SIM_MODE_PARAM_ROWS) return fail(SIM_EINVAL, "bad mode %d", mode);
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    // layout
    std::vector<int> d(3 * (size_t)P);
    std::vector<int64_t> voff(P + 1, 0), moff(P + 1, 0), soff(P + 1, 0);
    int max_corner = 0;
    int64_t max_sc = 0;
    for (int r = 0; r < P; ++r) {
        for (int a = 0; a < 3; ++a) {
            int v = dims[3 * r + a];
            if (v < 1 || v > kMaxAxis) return fail(SIM_EINVAL, "robot %d: dims must be in 1..%d", r, kMaxAxis);
            d[3 * r + a] = v;
        }
        const int nx = d[3 * r], ny = d[3 * r + 1], nz = d[3 * r + 2];
        const int corners = (nx + 1) * (ny + 1) * (nz + 1);
        const int64_t sc = full_springs(nx, ny, nz);
        voff[r + 1] = voff[r] + (int64_t)nx * ny * nz;
        moff[r + 1] = moff[r] + corners;
        soff[r + 1] = soff[r] + sc;
        max_corner = std::max(max_corner, corners);
        max_sc = std::max(max_sc, sc);
    }
    if ((mode == SIM_MODE_MLP || mode == SIM_MODE_PARAM_ROWS) && P > 0) {
        for (int r = 1; r < P; ++r)
            if (d[3 * r] != d[0] || d[3 * r + 1] != d[1] || d[3 * r + 2] != d[2])
                return fail(SIM_EINVAL, "this mode needs one grid shape for all robots");
        if (mode == SIM_MODE_MLP && !B) return fail(SIM_EINVAL, "MLP mode needs the encoding matrix B");
    }
    if (P > 0 && !genomes) return fail(SIM_EINVAL, "null genomes");
    const int64_t V = voff[P], Mc = moff[P], Sc = soff[P];
    const bool packed = max_corner <= kResidentMaxCorner;
    if (!packed && ctx->p.path == SIM_PATH_RESIDENT)
        return fail(SIM_EINVAL, "robots with more than %d corners need the streamed path", kResidentMaxCorner);
    if (mode == SIM_MODE_MLP && !packed)
        return fail(SIM_EINVAL, "MLP decoding supports grids of at most %d corners", kResidentMaxCorner);
    // host-side validation of host materials
    if (mem == SIM_MEM_HOST && (mode == SIM_MODE_MATERIALS || mode == SIM_MODE_PARAMS || mode == SIM_MODE_PARAM_ROWS)) {
        const uint8_t* m = mode == SIM_MODE_MATERIALS ? (const uint8_t*)genomes
                           : mode == SIM_MODE_PARAMS  ? ((const sim_voxel_params*)genomes)->mat
                                                      : ((const sim_param_rows*)genomes)->mat;
        if (V > 0 && !m) return fail(SIM_EINVAL, "null materials");
        for (int64_t i = 0; i < V; ++i)
            if (m[i] >= kNumMat) return fail(SIM_EINVAL, "material id %d at voxel %lld", (int)m[i], (long long)i);
    }
    if (mode == SIM_MODE_PARAMS) {
        const sim_voxel_params* vp = (const sim_voxel_params*)genomes;
        if (V > 0 && (!vp->mat || !vp->w || !vp->kappa || !vp->phi))
            return fail(SIM_EINVAL, "null per-voxel parameter array");
    }
    // buffers
    VX_CK(ctx->d_dims.ensure(3 * (size_t)P));
    VX_CK(ctx->d_voff.ensure(P + 1)); VX_CK(ctx->d_moff.ensure(P + 1)); VX_CK(ctx->d_soff.ensure(P + 1));
    VX_CK(ctx->d_tmp_off.ensure(P + 1));
    VX_CK(ctx->d_nm.ensure(P)); VX_CK(ctx->d_ns.ensure(P)); VX_CK(ctx->d_lpt.ensure(P));
    VX_CK(ctx->d_queue.ensure(2)); VX_CK(ctx->d_status.ensure(4));
    VX_CK(ctx->d_mat_raw.ensure(V)); VX_CK(ctx->d_mat.ensure(V));
    VX_CK(ctx->d_w.ensure(V)); VX_CK(ctx->d_kappa.ensure(V)); VX_CK(ctx->d_phi.ensure(V));
    VX_CK(ctx->d_label.ensure(V)); VX_CK(ctx->d_count.ensure(V));
    VX_CK(ctx->d_corner_mass.ensure(Mc)); VX_CK(ctx->d_mass_corner.ensure(Mc));
    VX_CK(ctx->d_sab.ensure(Sc)); VX_CK(ctx->d_sp.ensure(Sc));
    if (packed) VX_CK(ctx->d_spack.ensure(Sc));
    ctx->have_pack = packed;
    VX_CK(ctx->d_x0.ensure(Mc)); VX_CK(ctx->d_x.ensure(Mc)); VX_CK(ctx->d_v.ensure(Mc));
    VX_CK(ctx->d_cflags.ensure(Mc)); VX_CK(ctx->d_prm.ensure(39 * (size_t)Mc));
    VX_CK(ctx->d_x0c.ensure(P)); VX_CK(ctx->d_keys.ensure(P)); VX_CK(ctx->d_fit.ensure(P));
    ctx->dims = d; ctx->voff = voff; ctx->moff = moff; ctx->soff = soff;
    ctx->P = P; ctx->V_tot = V; ctx->M_cap = Mc; ctx->S_cap = Sc;
    ctx->max_corner = max_corner; ctx->max_spring_cap = max_sc;
    ctx->have_pop = false;
    if (P > 0) {
        VX_CK(cudaMemcpyAsync(ctx->d_dims.p, d.data(), sizeof(int) * 3 * P, cudaMemcpyHostToDevice, s));
        VX_CK(cudaMemcpyAsync(ctx->d_voff.p, voff.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
        VX_CK(cudaMemcpyAsync(ctx->d_moff.p, moff.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
        VX_CK(cudaMemcpyAsync(ctx->d_soff.p, soff.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
    }
    VX_CK(cudaMemsetAsync(ctx->d_status.p, 0, 4 * sizeof(int), s));
    ctx->host_genome_floats = 0;
    ctx->imp_active = false;        // imposed contact modes belong to the previous population
    ctx->imp_n = 0;
    ctx->imp_off.clear();
    ctx->imp_table.clear();
    const MatConst mc = ctx->matconst();
    // decode
    if (P > 0) {
        if (mode == SIM_MODE_MATERIALS) {
            const uint8_t* src = (const uint8_t*)genomes;
            if (mem == SIM_MEM_HOST) {
                VX_CK(ctx->d_in_u8.ensure(V));
                if (sim_status st = copy_in(genomes, V, mem, ctx->d_in_u8.p, s)) return st;
                src = ctx->d_in_u8.p;
            }
            VX_LAUNCH(ctx, launch_decode_materials(src, V, mc, ctx->d_mat_raw.p, ctx->d_w.p, ctx->d_kappa.p,
                                          ctx->d_phi.p, ctx->d_status.p, s));
        } else if (mode == SIM_MODE_LOGITS) {
            const float* src = (const float*)genomes;
            if (mem == SIM_MEM_HOST) {
                VX_CK(ctx->d_in_f32.ensure(5 * (size_t)V));
                if (sim_status st = copy_in(genomes, sizeof(float) * 5 * V, mem, ctx->d_in_f32.p, s)) return st;
                src = ctx->d_in_f32.p;
                ctx->host_genome_floats = 5 * V;
            }
            VX_LAUNCH(ctx, launch_decode_logits(src, V, mc, ctx->d_mat_raw.p, ctx->d_w.p, ctx->d_kappa.p,
                                       ctx->d_phi.p, s));
        } else if (mode == SIM_MODE_PARAMS) {
            const sim_voxel_params* vp = (const sim_voxel_params*)genomes;
            const uint8_t* m = vp->mat;
            const float *w = vp->w, *k = vp->kappa, *ph = vp->phi;
            if (mem == SIM_MEM_HOST) {
                VX_CK(ctx->d_in_u8.ensure(V));
                VX_CK(ctx->d_in_f32.ensure(V)); VX_CK(ctx->d_in_f32b.ensure(V)); VX_CK(ctx->d_in_f32c.ensure(V));
                if (sim_status st = copy_in(m, V, mem, ctx->d_in_u8.p, s)) return st;
                if (sim_status st = copy_in(w, 4 * V, mem, ctx->d_in_f32.p, s)) return st;
                if (sim_status st = copy_in(k, 4 * V, mem, ctx->d_in_f32b.p, s)) return st;
                if (sim_status st = copy_in(ph, 4 * V, mem, ctx->d_in_f32c.p, s)) return st;
                m = ctx->d_in_u8.p; w = ctx->d_in_f32.p; k = ctx->d_in_f32b.p; ph = ctx->d_in_f32c.p;
            }
            VX_LAUNCH(ctx, launch_decode_params(m, w, k, ph, V, ctx->d_mat_raw.p, ctx->d_w.p, ctx->d_kappa.p,
                                       ctx->d_phi.p, ctx->d_status.p, s));
        } else if (mode == SIM_MODE_PARAM_ROWS) {
            const sim_param_rows* pr = (const sim_param_rows*)genomes;
            const uint8_t* m = pr->mat;
            const float* rows = pr->rows;
            if (V > 0 && (!m || !rows)) return fail(SIM_EINVAL, "null materials or rows");
            if (mem == SIM_MEM_HOST) {
                VX_CK(ctx->d_in_u8.ensure(V));
                VX_CK(ctx->d_in_f32.ensure(3 * (size_t)V));
                if (sim_status st = copy_in(m, V, mem, ctx->d_in_u8.p, s)) return st;
                if (sim_status st = copy_in(rows, 12 * V, mem, ctx->d_in_f32.p, s)) return st;
                m = ctx->d_in_u8.p; rows = ctx->d_in_f32.p;
                ctx->host_genome_floats = 3 * V;
            }
            VX_LAUNCH(ctx, launch_decode_param_rows(m, rows, V / P, V, ctx->d_mat_raw.p, ctx->d_w.p,
                                                    ctx->d_kappa.p, ctx->d_phi.p, ctx->d_status.p, s));
        } else {
            const int Q = d[0] * d[1] * d[2];
            const float* gsrc = (const float*)genomes;
            const float* bsrc = B;
            if (mem == SIM_MEM_HOST) {
                VX_CK(ctx->d_in_f32.ensure((size_t)P * kGenome));
                VX_CK(ctx->d_in_f32b.ensure(kPeRows * 3));
                if (sim_status st = copy_in(genomes, sizeof(float) * (size_t)P * kGenome, mem, ctx->d_in_f32.p, s)) return st;
                if (sim_status st = copy_in(B, sizeof(float) * kPeRows * 3, mem, ctx->d_in_f32b.p, s)) return st;
                gsrc = ctx->d_in_f32.p;
                bsrc = ctx->d_in_f32b.p;
                ctx->host_genome_floats = (int64_t)P * kGenome;
            }
            VX_CK(ctx->d_pe.ensure((size_t)Q * kPeDim * 2));
            VX_LAUNCH(ctx, launch_pe_table(d[0], d[1], d[2], bsrc, ctx->d_pe.p, s));
            if (ctx->p.mlp_kernel == SIM_MLP_SIMT)
                VX_LAUNCH(ctx, launch_mlp_query_simt(P, Q, ctx->d_pe.p, gsrc, mc, ctx->d_mat_raw.p, ctx->d_w.p,
                                                     ctx->d_kappa.p, ctx->d_phi.p, s));
            else
                VX_LAUNCH(ctx, launch_mlp_query(P, Q, ctx->d_pe.p, gsrc, mc, ctx->d_mat_raw.p, ctx->d_w.p,
                                                ctx->d_kappa.p, ctx->d_phi.p, ctx->d_status.p + 1,
                                                ctx->num_sms, s));
        }
        // topology
        VX_LAUNCH(ctx, launch_topology(ctx->view(), ctx->d_mat_raw.p, ctx->d_mat.p, ctx->d_w.p, ctx->d_kappa.p,
                              ctx->d_phi.p, mc, ctx->p.edge, ctx->d_label.p, ctx->d_count.p,
                              ctx->d_corner_mass.p, ctx->d_mass_corner.p, ctx->d_sab.p, ctx->d_sp.p,
                              packed ? ctx->d_spack.p : nullptr, ctx->d_cflags.p, ctx->d_prm.p,
                              ctx->d_x0.p, ctx->d_x.p, ctx->d_v.p,
                              ctx->d_x0c.p, ctx->d_status.p, 0, s));
        // longest-first processing order (by spring count, ties by index)
        k_spring_keys<<<(P + 255) / 256, 256, 0, s>>>(ctx->d_ns.p, P, ctx->d_keys.p);
        VX_LAUNCH(ctx, cudaGetLastError());
        VX_LAUNCH(ctx, launch_evo_rank(ctx->d_keys.p, P, ctx->d_lpt.p, s));
        // the mass counts order the work queue (longest first); the plan is built on the host
        ctx->mass_count.assign(P, 0);
        ctx->spring_count.assign(P, 0);
        VX_CK(cudaMemcpyAsync(ctx->mass_count.data(), ctx->d_nm.p, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        VX_CK(cudaMemcpyAsync(ctx->spring_count.data(), ctx->d_ns.p, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        int32_t words[4] = {0, 0, 0, 0};
        VX_CK(cudaMemcpyAsync(words, ctx->d_status.p, sizeof(words), cudaMemcpyDeviceToHost, s));
        VX_CK(cudaStreamSynchronize(s));
        if (sim_status st = status_from_words(words)) return st;
        if (sim_status st = build_work_items(ctx)) return st;
    }
    ctx->step = 0;
    ctx->rec_valid = false;
    ctx->drop_graph();
    ctx->have_pop = true;
    return SIM_OK;
}

// Default kind of a size class: the lattice kernel up to its block size, then the atomic
// resident kernel while the robot's state fits one SM, then the streamed path.
static bool is_lattice(int kind) { return kind == kKindLattice || kind == kKindLatticeCompact; }

// CTAs per cluster for a robot on the cluster lattice kernel: the fewest slabs of whole corner
// layers with at most 768 corners each; 0 when a layer alone is too large or more than 8 slabs
// would be needed, 1 when the robot fits one block.
static int cluster_q(int nx, int ny, int nz)
{
    const int XY = (nx + 1) * (ny + 1), Z = nz + 1, T = cluster_max_threads();
    if (XY > T) return 0;
    const int Lmax = T / XY;
    const int q = (Z + Lmax - 1) / Lmax;
    return q <= 8 ? q : 0;
}

// The lattice variant a size class takes before any tuning: the requested one, else the
// per-corner kernel (measured faster than the compacted one on every workload tried: uniform,
// Bernoulli 0.3 to 1.0 and MLP-decoded 8x8x8 grids, uneven populations).
static int lattice_default(const voxsim_ctx* ctx)
{
    return ctx->p.lattice == SIM_LATTICE_COMPACT ? kKindLatticeCompact : kKindLattice;
}

static void default_choices(voxsim_ctx* ctx)
{
    const size_t budget = ctx->smem_optin > 2048 ? ctx->smem_optin - 1024 : ctx->smem_optin;
    for (int k = 0; k < kNumClasses; ++k) {
        const int C = std::min(kClassCorners[k], kResidentMaxCorner);
        const bool fits = resident_smem_bytes(C, 0, SIM_ACC_ATOMIC) <= budget && kClassCorners[k] <= kResidentMaxCorner;
        // robots of up to 768 corners: one lattice block; larger: the lattice kernel in
        // mass-sized thread groups for those of at most 768 masses (measured 1.87x the atomic
        // kernel's rate on the uneven population's 824 such robots: 9.1 against 17.0 ms for 500
        // steps), the atomic kernel for the others while it fits (measured ahead of the cluster
        // of lattice blocks, 47 against 63 ms on the uneven population's large robots), else
        // streamed.  Bit-reproducible stepping takes the cluster of lattice blocks for robots of
        // more than 768 masses (ahead of the streamed path: 63 against 80 ms).
        int kind = k < 6 ? lattice_default(ctx) : (fits ? kKindMassGroups : kKindStreamed);
        if (kind == kKindAtomic && ctx->p.accumulate == SIM_ACC_GATHER) kind = kKindCluster;
        if (kind == kKindMassGroups && ctx->p.accumulate == SIM_ACC_ATOMIC) kind = kKindAtomic;
        if (is_lattice(kind) && ctx->p.accumulate == SIM_ACC_ATOMIC) kind = kKindAtomic;
        ctx->class_kind[k] = kind;
        ctx->class_threads[k] = 0;
    }
}

// Execution plan of the population from the per-class choices:
//   lattice: work items of robots grouped by corner count into 64..768-thread slots of a
//   768-thread block (several small robots per block), largest class first, robots by
//   descending corner count (longest processing time first);
//   atomic: one persistent launch per thread count, robots longest first;
//   streamed: the rest.
// Everything is known from the grid shapes, so no device data is read.
static sim_status build_work_items(voxsim_ctx* ctx, const std::vector<int>* subset)
{
    static const int kSlot[6] = {64, 128, 192, 256, 384, 768};
    const int block = lattice_max_threads();
    ++ctx->items_version;
    if (!ctx->tuned) default_choices(ctx);
    ctx->has_split = false;
    ctx->max_big_corner = 0;
    ctx->max_big_spring_cap = 0;
    ctx->atomic_groups.clear();
    if (ctx->p.path == SIM_PATH_PLAIN) {       // every robot on the baseline kernels
        ctx->n_items = ctx->n_items_corner = ctx->n_big = ctx->n_stream = ctx->n_cluster = 0;
        ctx->cluster_groups.clear();
        VX_CK(ctx->d_plain_f.ensure(3 * (size_t)ctx->M_cap));
        VX_CK(cudaMemsetAsync(ctx->d_plain_f.p, 0, sizeof(float) * 3 * (size_t)ctx->M_cap, ctx->stream));
        return SIM_OK;
    }
    const size_t budget = ctx->smem_optin > 2048 ? ctx->smem_optin - 1024 : ctx->smem_optin;
    const bool damped = ctx->stepconst().damped != 0;
    std::vector<std::vector<std::pair<int, int>>> lattice(6), lattice_sp(6);
    std::vector<std::pair<int, std::pair<int, int>>> atomic;   // (threads, (-corners, robot))
    std::vector<int> streamed;
    std::vector<std::pair<int, int>> clustered;                  // (q, robot)
    std::vector<int> mass_groups;                                // larger robots in mass-sized groups
    ctx->max_stream_corner = 0;
    const int nrob = subset ? (int)subset->size() : ctx->P;
    for (int ri = 0; ri < nrob; ++ri) {
        const int r = subset ? (*subset)[ri] : ri;
        const int nx = ctx->dims[3 * r], ny = ctx->dims[3 * r + 1], nz = ctx->dims[3 * r + 2];
        const int C = (nx + 1) * (ny + 1) * (nz + 1);
        const int k = class_of(C);
        const bool fits_sm = C <= kResidentMaxCorner && resident_smem_bytes(C, 0, SIM_ACC_ATOMIC) <= budget;
        const int q = cluster_q(nx, ny, nz);            // >= 2: the cluster lattice kernel can take it
        int kind = ctx->class_kind[k];
        // SIM_LATTICE_PACKED asks for mass-sized groups wherever a robot fits them
        if (ctx->p.lattice == SIM_LATTICE_PACKED && C > block) kind = kKindMassGroups;
        // robots of more than a block's corners but at most a block's masses can run on the
        // lattice kernel in mass-sized thread groups (deterministic); else the class's atomic
        // alternative
        if (kind == kKindMassGroups) {
            const bool known = (int)ctx->mass_count.size() == ctx->P;
            const int M = known ? ctx->mass_count[r] : 0;
            const int T = (M + 31) / 32 * 32;
            const size_t need = sizeof(float4) * ((damped ? 2 : 1) * (size_t)C + 13 * (size_t)T + 32);
            if (C <= block) kind = lattice_default(ctx);
            else if (known && M >= 1 && T <= block && need <= budget && ctx->ckpt_every == 0 &&
                     ctx->p.accumulate != SIM_ACC_ATOMIC && ctx->p.path != SIM_PATH_STREAMED && !ctx->imp_active) {
                mass_groups.push_back(r);
                continue;
            } else {
                kind = ctx->p.accumulate == SIM_ACC_GATHER ? kKindCluster : kKindAtomic;
            }
        }
        if (ctx->p.path == SIM_PATH_STREAMED) kind = kKindStreamed;
        else if (ctx->p.accumulate == SIM_ACC_ATOMIC && (is_lattice(kind) || kind == kKindCluster)) kind = kKindAtomic;
        else if (ctx->p.accumulate == SIM_ACC_GATHER && kind == kKindAtomic) kind = k < 6 ? lattice_default(ctx) : kKindCluster;
        // what the robot's size allows
        if (is_lattice(kind) && C > block) kind = q >= 2 ? kKindCluster : kKindAtomic;
        if (kind == kKindCluster && q < 2)
            kind = C <= block ? lattice_default(ctx)
                              : (fits_sm && ctx->p.accumulate != SIM_ACC_GATHER ? kKindAtomic : kKindStreamed);
        if (kind == kKindAtomic && !fits_sm) kind = q >= 2 && ctx->p.accumulate != SIM_ACC_ATOMIC ? kKindCluster : kKindStreamed;
        // the adjoint replays large robots on the streamed path
        if ((kind == kKindAtomic || kind == kKindCluster) && ctx->ckpt_every > 0) kind = kKindStreamed;
        if (kind == kKindStreamed && ctx->p.path == SIM_PATH_RESIDENT) {
            if (C <= block && ctx->p.accumulate != SIM_ACC_ATOMIC) kind = lattice_default(ctx);
            else if (q >= 2 && ctx->p.accumulate != SIM_ACC_ATOMIC && ctx->ckpt_every == 0) kind = kKindCluster;
            else if (fits_sm && ctx->p.accumulate != SIM_ACC_GATHER) kind = kKindAtomic;
            else return fail(SIM_EINVAL, "robot %d (%d corners) does not fit the resident path", r, C);
        }
        // while contact modes are imposed every robot that fits a lattice block runs on it
        if (ctx->imp_active && C <= block && ctx->p.accumulate != SIM_ACC_ATOMIC) kind = kKindLattice;
        // a requested variant wins over the class choice; the direction-compacted one needs the list
        if (kind == kKindLattice && ctx->p.lattice == SIM_LATTICE_COMPACT) kind = kKindLatticeCompact;
        if (kind == kKindLatticeCompact &&
            (ctx->p.lattice == SIM_LATTICE_CORNER || ctx->p.lattice == SIM_LATTICE_PACKED || !ctx->have_pack ||
             ctx->imp_active))
            kind = kKindLattice;
        if (kind == kKindAtomic && ctx->p.accumulate == SIM_ACC_GATHER)
            return fail(SIM_EINVAL, "bit-reproducible stepping supports robots of at most %d corners on the resident path", block);
        if (is_lattice(kind)) {
            int slot = 0;
            while (kSlot[slot] < C) ++slot;
            // longest first: by mass count when known (the step's cost follows the masses), else corners
            const int key = (int)ctx->mass_count.size() == ctx->P ? ctx->mass_count[r] : C;
            (kind == kKindLattice ? lattice : lattice_sp)[slot].push_back({-key, r});
        } else if (kind == kKindCluster) {
            clustered.push_back({cluster_q(nx, ny, nz), r});
        } else if (kind == kKindAtomic) {
            int threads = ctx->class_threads[k] > 0 ? ctx->class_threads[k] : ctx->p.threads;
            if (threads <= 0) {
                const int64_t sc = full_springs(nx, ny, nz);
                threads = sc <= 1536 ? 256 : (sc <= 6144 ? 512 : 1024);
            }
            threads = std::max(32, std::min(1024, (threads + 31) / 32 * 32));
            // longest first: by spring count when known (a thread per spring), else corners
            const int key = (int)ctx->spring_count.size() == ctx->P ? ctx->spring_count[r] : C;
            atomic.push_back({threads, {-key, r}});
        } else {
            streamed.push_back(r);
            ctx->max_stream_corner = std::max(ctx->max_stream_corner, C);
        }
    }
    std::vector<int4> items;
    std::vector<int> robots;
    // robots per block: as many as the slots hold when the population is large, fewer when that
    // would leave SMs idle (a population of 30 small robots runs on 30 SMs, not 10)
    size_t n_lattice = 0;
    for (int k = 0; k < 6; ++k) n_lattice += lattice[k].size() + lattice_sp[k].size();
    const int spread = (int)std::max<size_t>(1, n_lattice / (size_t)std::max(1, ctx->num_sms));
    for (int variant = 0; variant < 2; ++variant) {
        if (variant == 1) ctx->n_items_corner = (int)items.size();
        for (int k = 5; k >= 0; --k) {
            auto& v = variant == 0 ? lattice[k] : lattice_sp[k];
            std::sort(v.begin(), v.end());
            const int per = std::min(block / kSlot[k], spread);
            // a robot alone in its block gets a second thread per corner (split item) when the
            // slot allows and the springs have dashpots: its step's chain of spring evaluations
            // is cut from 13 to 7 (measured -14 % on the paper's 30 robots 5x5x5; without
            // dashpots the split measured from -13 % to +27 %, so it is not used there)
            const bool split = variant == 0 && per == 1 && 2 * kSlot[k] <= block && damped;
            for (size_t i = 0; i < v.size(); i += per) {
                const int n = (int)std::min<size_t>(per, v.size() - i);
                items.push_back(make_int4((int)robots.size(), n, split ? 2 * kSlot[k] : kSlot[k],
                                          split ? 2 : variant));
                for (int j = 0; j < n; ++j) robots.push_back(v[i + j].second);
            }
            if (split && !v.empty()) ctx->has_split = true;
        }
    }
    // the per-corner kernel's compile-time 8 x 8 x 8 instantiation applies when every one of its
    // items is a single robot of that grid in a 768-thread slot
    ctx->corner_cube8 = ctx->n_items_corner > 0;
    for (int i = 0; i < ctx->n_items_corner && ctx->corner_cube8; ++i) {
        const int4 it = items[i];
        const int r = robots[it.x];
        ctx->corner_cube8 = it.y == 1 && it.z == 768 && it.w == 0 && ctx->dims[3 * r] == 8 &&
                            ctx->dims[3 * r + 1] == 8 && ctx->dims[3 * r + 2] == 8;
    }
    if (sim_status st = build_packed_items(ctx, lattice, mass_groups, damped)) return st;
    std::sort(atomic.begin(), atomic.end());
    std::vector<int> big;
    for (size_t i = 0; i < atomic.size();) {
        voxsim_ctx::AtomicGroup g{atomic[i].first, (int)big.size(), 0, 0, 0};
        for (; i < atomic.size() && atomic[i].first == g.threads; ++i) {
            const int r = atomic[i].second.second;
            big.push_back(r);
            g.max_corner = std::max(g.max_corner, (ctx->dims[3 * r] + 1) * (ctx->dims[3 * r + 1] + 1) *
                                                      (ctx->dims[3 * r + 2] + 1));
            g.max_spring_cap = std::max(g.max_spring_cap, full_springs(ctx->dims[3 * r], ctx->dims[3 * r + 1], ctx->dims[3 * r + 2]));
        }
        g.count = (int)big.size() - g.first;
        ctx->max_big_corner = std::max(ctx->max_big_corner, g.max_corner);
        ctx->max_big_spring_cap = std::max(ctx->max_big_spring_cap, g.max_spring_cap);
        ctx->atomic_groups.push_back(g);
    }
    std::sort(clustered.begin(), clustered.end());
    std::vector<int> cl_robots;
    ctx->cluster_groups.clear();
    for (size_t i = 0; i < clustered.size();) {
        voxsim_ctx::ClusterGroup g{clustered[i].first, (int)cl_robots.size(), 0};
        for (; i < clustered.size() && clustered[i].first == g.q; ++i) cl_robots.push_back(clustered[i].second);
        g.count = (int)cl_robots.size() - g.first;
        ctx->cluster_groups.push_back(g);
    }
    ctx->n_cluster = (int)cl_robots.size();
    ctx->n_items = (int)items.size();
    ctx->n_big = (int)big.size();
    ctx->n_stream = (int)streamed.size();
    ctx->stream_robots = streamed;
    ctx->stream_cube40 = !streamed.empty();
    for (int r : streamed)
        ctx->stream_cube40 = ctx->stream_cube40 && ctx->dims[3 * r] == 40 && ctx->dims[3 * r + 1] == 40 &&
                             ctx->dims[3 * r + 2] == 40;
    cudaStream_t s = ctx->stream;
    VX_CK(ctx->d_queue.ensure(2 + ctx->atomic_groups.size()));
    if (!streamed.empty()) {
        VX_CK(ctx->d_stream.ensure(streamed.size()));
        VX_CK(cudaMemcpyAsync(ctx->d_stream.p, streamed.data(), sizeof(int) * streamed.size(),
                              cudaMemcpyHostToDevice, s));
        // both state buffers start equal (corners without a mass are never rewritten)
        VX_CK(ctx->d_x_alt.ensure(ctx->M_cap));
        VX_CK(ctx->d_v_alt.ensure(ctx->M_cap));
        VX_CK(cudaMemcpyAsync(ctx->d_x_alt.p, ctx->d_x.p, sizeof(float4) * ctx->M_cap, cudaMemcpyDeviceToDevice, s));
        VX_CK(cudaMemcpyAsync(ctx->d_v_alt.p, ctx->d_v.p, sizeof(float4) * ctx->M_cap, cudaMemcpyDeviceToDevice, s));
    }
    VX_CK(ctx->d_items.ensure(items.size()));
    VX_CK(ctx->d_progress.ensure(items.size()));
    VX_CK(ctx->d_item_robots.ensure(robots.size()));
    VX_CK(ctx->d_big.ensure(big.size()));
    if (!items.empty()) {
        VX_CK(cudaMemcpyAsync(ctx->d_items.p, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s));
        VX_CK(cudaMemcpyAsync(ctx->d_item_robots.p, robots.data(), sizeof(int) * robots.size(), cudaMemcpyHostToDevice, s));
    }
    if (!big.empty())
        VX_CK(cudaMemcpyAsync(ctx->d_big.p, big.data(), sizeof(int) * big.size(), cudaMemcpyHostToDevice, s));
    VX_CK(ctx->d_cluster.ensure(cl_robots.size()));
    if (!cl_robots.empty())
        VX_CK(cudaMemcpyAsync(ctx->d_cluster.p, cl_robots.data(), sizeof(int) * cl_robots.size(),
                              cudaMemcpyHostToDevice, s));
    // the host vectors are copied from pageable memory: wait so they may go out of scope
    VX_CK(cudaStreamSynchronize(s));
    ctx->drop_graph();
    return SIM_OK;
}

// Mass-packed plan of the per-corner lattice robots (SIM_LATTICE_PACKED): groups of
// T = (masses rounded up to a warp) threads, packed first-fit by decreasing T into 768-thread
// blocks under the shared-memory budget (C displacements, C velocities with dashpots, 13 T plane
// entries and 32 rows for absent springs per group) and at most 15 groups (named barriers
// 1..15).  When the packed blocks would not fill every SM, the thread capacity of a block
// shrinks so that the work spreads over all of them.
static sim_status build_packed_items(voxsim_ctx* ctx, const std::vector<std::vector<std::pair<int, int>>>& lattice,
                                     const std::vector<int>& mass_groups, bool damped)
{
    ctx->n_pitems = 0;
    ctx->pitems_cover_corner = false;
    ctx->pitem_smem = 0;
    const bool masses_known = (int)ctx->mass_count.size() == ctx->P;
    // the per-corner robots join the packed plan only when asked for: measured slower than the
    // one-robot-per-slot kernel on the workloads tried (its address arithmetic adds 22 %
    // instructions, and the slot kernel's throughput is bound by issue and the shared-memory
    // pipe rather than by its idle warps); robots of more than a block's corners come here when
    // their size class chose mass-sized groups
    // By default they join once the population has thinned: when the robots' masses fill less
    // than 55 % of the threads of their corner-sized slots, packing them pays (measured on the
    // MLP population's 10 generations: -17 % at generations 8 and 9, 51-53 % filled; even at 57 %;
    // +10 to +22 % while 62-83 % filled).
    bool thin = false;
    if (masses_known && ctx->p.lattice == SIM_LATTICE_AUTO) {
        static const int kSlotT[6] = {64, 128, 192, 256, 384, 768};
        int64_t used = 0, slots = 0;
        size_t n = 0;
        for (int k = 0; k < 6; ++k)
            for (const auto& e : lattice[k]) {
                used += ctx->mass_count[e.second];
                slots += kSlotT[k];
                ++n;
            }
        thin = n > (size_t)ctx->num_sms && slots > 0 && (double)used < 0.55 * (double)slots;
    }
    const bool corner_too = masses_known && (ctx->p.lattice == SIM_LATTICE_PACKED || thin) && !ctx->has_split &&
                            !ctx->imp_active;
    struct Grp { int T, C, r; };
    std::vector<Grp> gs;
    int64_t sumT = 0;
    int maxT = 32;
    auto add = [&](int r) {
        const int M = ctx->mass_count[r];
        if (M <= 0) return;                             // nothing to step
        const int C = (ctx->dims[3 * r] + 1) * (ctx->dims[3 * r + 1] + 1) * (ctx->dims[3 * r + 2] + 1);
        const int T = (M + 31) / 32 * 32;
        gs.push_back({T, C, r});
        sumT += T;
        maxT = std::max(maxT, T);
    };
    if (corner_too)
        for (const auto& v : lattice)
            for (const auto& e : v) add(e.second);
    for (int r : mass_groups) add(r);
    ctx->pitems_cover_corner = corner_too;
    if (gs.empty()) { ctx->pitems_cover_corner = false; return SIM_OK; }
    std::sort(gs.begin(), gs.end(), [](const Grp& a, const Grp& b) {
        return a.T != b.T ? a.T > b.T : (a.C != b.C ? a.C > b.C : a.r < b.r);
    });
    const int block = lattice_max_threads();
    const size_t budget = ctx->smem_optin > 2048 ? ctx->smem_optin - 1024 : ctx->smem_optin;
    int cap = block;
    if (sumT < (int64_t)block * ctx->num_sms) {
        const int64_t per = (sumT + ctx->num_sms - 1) / ctx->num_sms;
        cap = (int)std::max<int64_t>(maxT, (per + 31) / 32 * 32);
    }
    auto need = [&](const Grp& g) {
        return sizeof(float4) * ((damped ? 2 : 1) * (size_t)g.C + 13 * (size_t)g.T + 32);
    };
    struct Bin { int threads; size_t smem; std::vector<int> members; };
    std::vector<Bin> bins;
    for (int i = 0; i < (int)gs.size(); ++i) {
        const size_t b = need(gs[i]);
        if (b > budget) return fail(SIM_EINVAL, "robot %d does not fit a lattice block", gs[i].r);
        Bin* home = nullptr;
        for (Bin& bin : bins)
            if (bin.threads + gs[i].T <= cap && bin.smem + b <= budget && bin.members.size() < 15) { home = &bin; break; }
        if (!home) { bins.push_back({0, 0, {}}); home = &bins.back(); }
        home->threads += gs[i].T;
        home->smem += b;
        home->members.push_back(i);
    }
    std::vector<int4> items, groups;
    for (const Bin& bin : bins) {
        items.push_back(make_int4((int)groups.size(), (int)bin.members.size(), 0, 0));
        int t0 = 0;
        size_t off = 0;
        for (int i : bin.members) {
            groups.push_back(make_int4(gs[i].r, t0, gs[i].T, (int)(off / sizeof(float4))));
            t0 += gs[i].T;
            off += need(gs[i]);
        }
        ctx->pitem_smem = std::max(ctx->pitem_smem, bin.smem);
    }
    VX_CK(ctx->d_pitems.ensure(items.size()));
    VX_CK(ctx->d_progress.ensure(items.size()));
    VX_CK(ctx->d_pgroups.ensure(groups.size()));
    VX_CK(cudaMemcpyAsync(ctx->d_pitems.p, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, ctx->stream));
    VX_CK(cudaMemcpyAsync(ctx->d_pgroups.p, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice, ctx->stream));
    // the host vectors go out of scope: the copies must have read them
    VX_CK(cudaStreamSynchronize(ctx->stream));
    ctx->n_pitems = (int)items.size();
    return SIM_OK;
}

// Next free event pair of the timing pool (grown on demand).
static sim_status timing_pair(voxsim_ctx* ctx, cudaEvent_t ev[2])
{
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
        cudaEvent_t e;
        VX_CK(cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
    }
    ev[0] = ctx->ev_pool[ctx->ev_used];
    ev[1] = ctx->ev_pool[ctx->ev_used + 1];
    ctx->ev_used += 2;
    return SIM_OK;
}

// Segments per item of the per-corner lattice launch: with more items than SMs, each item's n
// steps are split so that the queue holds about 64 units per SM (at least 256 steps each); the
// last wave then waits for one segment of the slowest items instead of one whole run.
static int lattice_segments(int items, int n, int sms)
{
    if (items <= sms || n < 512) return 1;
    const int want = (64 * sms + items - 1) / items, cap = n / 256;
    return std::max(1, std::min(want, cap));
}

// record: the call is sim_step_n's with checkpointing on (checkpoints, and the whole-trajectory
// records when they are kept, are written; every other caller steps without recording).
static sim_status step_lattice(voxsim_ctx* ctx, int n, bool record)
{
    if (ctx->n_items == 0 && ctx->n_pitems == 0) return SIM_OK;
    LatticeArgs a{};
    a.pv = ctx->view();
    a.corner_order = ctx->d_mass_corner.p;
    a.cflags = ctx->d_cflags.p;
    a.prm = ctx->d_prm.p;
    a.u = ctx->d_x.p;
    a.v = ctx->d_v.p;
    a.sc = ctx->d_sc.p;
    a.nsteps = n;
    a.c = ctx->stepconst();
    a.items = ctx->d_items.p;
    a.item_robots = ctx->d_item_robots.p;
    a.n_items = ctx->n_items;
    a.queue = ctx->d_queue.p;
    a.has_split = ctx->has_split ? 1 : 0;
    a.cube8 = ctx->corner_cube8 ? 1 : 0;
    ctx->imposed_args(a, ctx->step);
    if (record) {                               // (buffers sized by sim_step_n)
        a.ckpt_u = ctx->d_ckpt_u.p;
        a.ckpt_v = ctx->d_ckpt_v.p;
        a.ckpt_stride = ctx->M_cap;
        a.ckpt_every = ctx->ckpt_every;
        if (ctx->keep_records) {                // every step's record, for a replay-free backward
            a.rec_u = ctx->d_trec_u.p;
            a.rec_f = ctx->d_trec_f.p;
            a.rec_stride = (int64_t)ctx->M_cap;
        }
    }
    const int threads = lattice_max_threads();
    const size_t smem = sizeof(float4) * kLatticeSlotVec4 * (size_t)threads;
    VX_CK(cudaMemsetAsync(ctx->d_queue.p, 0, 2 * sizeof(int), ctx->stream));
    // per-corner variant: items [0, n_items_corner); direction-compacted variant: the rest
    const int n_corner = ctx->n_items_corner, n_spring = ctx->n_items - ctx->n_items_corner;
    const bool packed = ctx->n_pitems > 0 && !a.rec_u;
    if (packed) {
        // mass-sized groups: robots of more than a block's corners, and the per-corner robots
        // when the plan covers them (identical bits; checkpoints written alike)
        LatticeArgs b = a;
        b.items = ctx->d_pitems.p;
        b.groups = ctx->d_pgroups.p;
        b.n_items = ctx->n_pitems;
        b.queue = ctx->d_queue.p + 1;
        VX_CK(cudaMemsetAsync(b.queue, 0, sizeof(int), ctx->stream));
        // the same segmented queue as the per-corner launch below (undamped packed groups)
        const int nseg = !a.c.damped ? lattice_segments(ctx->n_pitems, n, ctx->num_sms) : 1;
        if (nseg > 1) {
            b.nseg = nseg;
            b.seg_steps = (n + nseg - 1) / nseg;
            b.progress = ctx->d_progress.p;
            b.status = ctx->d_status.p + 2;
            VX_CK(cudaMemsetAsync(b.progress, 0, sizeof(int) * ctx->n_pitems, ctx->stream));
        }
        VX_LAUNCH(ctx, launch_step_lattice_packed(b, std::min(ctx->n_pitems, ctx->num_sms), ctx->pitem_smem,
                                                  ctx->stream));
    }
    if (n_corner > 0 && !(packed && ctx->pitems_cover_corner)) {
        a.n_items = n_corner;
        // (segmented instantiations exist for the undamped per-corner steps without imposed
        // modes, recording only on 8 x 8 x 8 robots)
        const bool seg_ok = !a.imp_modes && !a.c.damped && (!a.rec_u || ctx->corner_cube8);
        const int nseg = seg_ok ? lattice_segments(n_corner, n, ctx->num_sms) : 1;
        if (nseg > 1) {
            a.nseg = nseg;
            a.seg_steps = (n + nseg - 1) / nseg;
            a.progress = ctx->d_progress.p;
            a.status = ctx->d_status.p + 2;
            VX_CK(cudaMemsetAsync(a.progress, 0, sizeof(int) * n_corner, ctx->stream));
        }
        VX_LAUNCH(ctx, launch_step_lattice(a, std::min(n_corner, ctx->num_sms), threads, smem, ctx->stream));
        a.nseg = 0;
    }
    if (n_spring > 0) {
        a.items = ctx->d_items.p + n_corner;
        a.n_items = n_spring;
        a.queue = ctx->d_queue.p + 1;
        if (packed) VX_CK(cudaMemsetAsync(a.queue, 0, sizeof(int), ctx->stream));   // reused after the packed launch
        a.spack = ctx->d_spack.p;
        VX_LAUNCH(ctx, launch_step_lattice(a, std::min(n_spring, ctx->num_sms), threads, smem, ctx->stream));
    }
    return SIM_OK;
}

// The cluster lattice kernel: one launch per cluster size, one cluster per robot.
static sim_status step_cluster(voxsim_ctx* ctx, int n)
{
    if (ctx->n_cluster == 0) return SIM_OK;
    ClusterArgs a{};
    a.pv = ctx->view();
    a.cflags = ctx->d_cflags.p;
    a.prm = ctx->d_prm.p;
    a.u = ctx->d_x.p;
    a.v = ctx->d_v.p;
    a.sc = ctx->d_sc.p;
    a.nsteps = n;
    a.c = ctx->stepconst();
    const size_t smem = sizeof(float4) * kLatticeSlotVec4 * (size_t)cluster_max_threads();
    for (const auto& g : ctx->cluster_groups) {
        a.robots = ctx->d_cluster.p + g.first;
        a.q = g.q;
        VX_LAUNCH(ctx, launch_step_cluster(a, g.count, smem, ctx->stream));
    }
    return SIM_OK;
}

// The atomic resident kernel: one persistent launch per thread count.
static sim_status step_resident(voxsim_ctx* ctx, int n)
{
    cudaStream_t s = ctx->stream;
    for (size_t gi = 0; gi < ctx->atomic_groups.size(); ++gi) {
        const voxsim_ctx::AtomicGroup& g = ctx->atomic_groups[gi];
        ResidentArgs a{};
        a.pv = ctx->view();
        a.spr_pack = ctx->d_spack.p;
        a.cflags = ctx->d_cflags.p;
        a.x = ctx->d_x.p;
        a.v = ctx->d_v.p;
        a.sc = ctx->d_sc.p;
        a.nsteps = n;
        a.c = ctx->stepconst();
        a.order = ctx->d_big.p + g.first;
        a.n_robots = g.count;
        a.queue = ctx->d_queue.p + 2 + gi;
        a.accumulate = SIM_ACC_ATOMIC;
        const int threads = g.threads;
        const int64_t sc = g.max_spring_cap;
        const size_t mass_bytes = resident_smem_bytes(g.max_corner, 0, a.accumulate);
        const size_t budget = ctx->smem_optin > 2048 ? ctx->smem_optin - 1024 : ctx->smem_optin;
        if (mass_bytes > budget) return fail(SIM_EINVAL, "robot too large for the resident path");
        int64_t spr_fit = (int64_t)((budget - mass_bytes) / sizeof(float4));
        // several blocks per SM when everything of the largest robot fits in a fraction of it
        int per_sm = 1;
        const size_t need = mass_bytes + sizeof(float4) * (size_t)sc;
        while (per_sm < 8 && need * (per_sm + 1) <= ctx->smem_optin && threads * (per_sm + 1) <= 2048)
            ++per_sm;
        if (per_sm > 1) spr_fit = sc;
        // a block with an SM to itself keeps its threads' first springs in tensor memory (the
        // 512 columns split over the warps of each lane quarter, 4 columns per spring)
        int tm_rec = 0, tm_cols = 0;
        if (per_sm == 1) {
            const int per_quarter = (threads / 32 + 3) / 4;
            tm_cols = (512 / per_quarter) & ~3;
            tm_rec = (int)std::min<int64_t>(tm_cols / 4, (sc + threads - 1) / threads);
        }
        a.tm_rec = tm_rec;
        a.tm_cols = tm_cols;
        a.max_mass = g.max_corner;
        a.max_spring_smem = (int)std::min<int64_t>(std::max<int64_t>(0, sc - (int64_t)tm_rec * threads), spr_fit);
        size_t smem = resident_smem_bytes(a.max_mass, a.max_spring_smem, a.accumulate);
        // a block that allocates the whole tensor memory must have its SM to itself: with the
        // springs moved out of shared memory it could otherwise share one with a second block,
        // which would wait for the first one's allocation until that block has drained the queue
        if (tm_rec > 0) smem = std::max(smem, (size_t)ctx->smem_optin / 2 + 4096);
        int grid = (int)std::min<int64_t>(g.count, (int64_t)ctx->num_sms * per_sm);
        if (grid < 1) grid = 1;
        VX_CK(cudaMemsetAsync(a.queue, 0, sizeof(int), s));
        VX_LAUNCH(ctx, launch_step_resident(a, grid, threads, smem, s));
    }
    return SIM_OK;
}

// The paper's organisation: for every step and robot, a spring launch and a mass launch.
static sim_status step_plain(voxsim_ctx* ctx, int n)
{
    cudaStream_t s = ctx->stream;
    std::vector<int32_t> M(ctx->P), S(ctx->P);
    if (sim_status st = sim_get_counts(ctx, M.data(), S.data())) return st;
    const StepConst c = ctx->stepconst();
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < ctx->P; ++r) {
            const int64_t mo = ctx->moff[r], so = ctx->soff[r];
            VX_CK(launch_step_plain_robot(ctx->d_sab.p + so, ctx->d_sp.p + so, ctx->d_mass_corner.p + mo,
                                          ctx->d_x.p + mo, ctx->d_v.p + mo, ctx->d_plain_f.p + 3 * mo, S[r], M[r],
                                          ctx->dims[3 * r], ctx->dims[3 * r + 1], ctx->d_sc.p, i, c, s));
            ctx->launches += (S[r] > 0) + (M[r] > 0);
        }
    return SIM_OK;
}

// Streamed robots: one launch per step, positions double-buffered; an odd number of steps
// leaves the newest positions in the alternate buffer, which are copied back per robot.
static sim_status enqueue_streamed(voxsim_ctx* ctx, int n, cudaStream_t s, bool record)
{
    StreamArgs a{};
    a.pv = ctx->view();
    a.cflags = ctx->d_cflags.p;
    a.prm = ctx->d_prm.p;
    a.sc = ctx->d_sc.p;
    a.c = ctx->stepconst();
    a.robots = ctx->d_stream.p;
    a.n_robots = ctx->n_stream;
    a.cube40 = ctx->stream_cube40 ? 1 : 0;
    const int K = record ? ctx->ckpt_every : 0;
    const bool keep = record && ctx->keep_records;
    for (int i = 0; i < n; ++i) {
        // the state at the start of every K-th step goes to its segment's checkpoint
        a.ckpt_u = K > 0 && i % K == 0 ? ctx->d_ckpt_u.p + (size_t)(i / K) * ctx->M_cap : nullptr;
        a.ckpt_v = K > 0 && i % K == 0 ? ctx->d_ckpt_v.p + (size_t)(i / K) * ctx->M_cap : nullptr;
        // and, when the whole trajectory is kept, every step's record
        a.rec_u = keep ? ctx->d_trec_u.p + (size_t)i * ctx->M_cap : nullptr;
        a.rec_f = keep ? ctx->d_trec_f.p + (size_t)i * ctx->M_cap : nullptr;
        a.u_in = (i & 1) ? ctx->d_x_alt.p : ctx->d_x.p;
        a.u_out = (i & 1) ? ctx->d_x.p : ctx->d_x_alt.p;
        a.v_in = (i & 1) ? ctx->d_v_alt.p : ctx->d_v.p;
        a.v_out = (i & 1) ? ctx->d_v.p : ctx->d_v_alt.p;
        VX_CK(launch_step_streamed(a, i, ctx->max_stream_corner, s));
    }
    if (n & 1)
        for (int r : ctx->stream_robots) {
            const size_t o = (size_t)ctx->moff[r], len = (size_t)(ctx->moff[r + 1] - ctx->moff[r]);
            VX_CK(cudaMemcpyAsync(ctx->d_x.p + o, ctx->d_x_alt.p + o, sizeof(float4) * len,
                                  cudaMemcpyDeviceToDevice, s));
            VX_CK(cudaMemcpyAsync(ctx->d_v.p + o, ctx->d_v_alt.p + o, sizeof(float4) * len,
                                  cudaMemcpyDeviceToDevice, s));
        }
    return SIM_OK;
}

// Streamed robots: one launch per step, positions double-buffered (an odd number of steps
// leaves the newest positions in the alternate buffer, copied back per robot).  The sequence is
// captured once into a CUDA graph per step count and replayed.
static sim_status step_streamed(voxsim_ctx* ctx, int n, bool record)
{
    if (ctx->n_stream == 0) return SIM_OK;
    cudaStream_t s = ctx->stream;
    const void* key = ctx->d_sc.p;   // the step table may move when it grows
    const void* ckpt = record ? (const void*)ctx->d_ckpt_u.p : nullptr;
    const void* trec = record && ctx->keep_records ? (const void*)ctx->d_trec_u.p : nullptr;
    if (!(ctx->stream_graph && ctx->stream_graph_n == n && ctx->stream_graph_key == key &&
          ctx->stream_graph_ckpt == ckpt && ctx->stream_graph_rec == trec &&
          ctx->stream_graph_every == (record ? ctx->ckpt_every : 0))) {
        ctx->drop_graph();
        if (!ctx->capture_stream) VX_CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        VX_CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        sim_status st = enqueue_streamed(ctx, n, ctx->capture_stream, record);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (st != SIM_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ctx->stream_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        ctx->stream_graph_n = n;
        ctx->stream_graph_key = key;
        ctx->stream_graph_ckpt = ckpt;
        ctx->stream_graph_rec = trec;
        ctx->stream_graph_every = record ? ctx->ckpt_every : 0;
    }
    VX_CK(cudaGraphLaunch(ctx->stream_graph, s));
    ctx->launches += n;
    return SIM_OK;
}

sim_status sim_step_n(voxsim_ctx* ctx, int32_t n_steps)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    if (n_steps < 0) return fail(SIM_EINVAL, "n_steps must be >= 0");
    if (n_steps == 0 || ctx->P == 0) return SIM_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    VX_CK(ctx->d_sc.ensure(n_steps));
    VX_LAUNCH(ctx, launch_sincos_table(2.0 * 3.141592653589793 * ctx->p.freq, ctx->p.dt, ctx->step, n_steps,
                              ctx->d_sc.p, s));
    if (ctx->ckpt_every > 0 && ctx->n_big > 0)
        return fail(SIM_EINVAL, "checkpointing needs the deterministic kernels (robots on the atomic kernel)");
    const bool record = ctx->ckpt_every > 0;
    // the buffers of the previous recorded call may be reallocated below: it is gone either way
    ctx->rec_valid = false;
    ctx->rec_full = false;
    if (record) {
        const int nseg = (n_steps + ctx->ckpt_every - 1) / ctx->ckpt_every;
        VX_CK(ctx->d_ckpt_u.ensure((size_t)nseg * ctx->M_cap));
        VX_CK(ctx->d_ckpt_v.ensure((size_t)nseg * ctx->M_cap));
        if (ctx->keep_records) {
            VX_CK(ctx->d_trec_u.ensure((size_t)n_steps * ctx->M_cap));
            VX_CK(ctx->d_trec_f.ensure((size_t)n_steps * ctx->M_cap));
        }
    }
    cudaEvent_t ev[2];
    if (sim_status st = timing_pair(ctx, ev)) return st;
    VX_CK(cudaEventRecord(ev[0], s));
    if (ctx->p.path == SIM_PATH_PLAIN) {
        if (sim_status st = step_plain(ctx, n_steps)) return st;
    } else {
        if (sim_status st = step_lattice(ctx, n_steps, record)) return st;
        if (sim_status st = step_cluster(ctx, n_steps)) return st;
        if (sim_status st = step_resident(ctx, n_steps)) return st;
        if (sim_status st = step_streamed(ctx, n_steps, record)) return st;
    }
    VX_CK(cudaEventRecord(ev[1], s));
    if (record) {
        ctx->rec_valid = true;
        ctx->rec_full = ctx->keep_records;
        ctx->rec_items_version = ctx->items_version;
        ctx->rec_step0 = ctx->step;
        ctx->rec_n = n_steps;
    }
    ctx->step += n_steps;
    return SIM_OK;
}

sim_status sim_fitness(voxsim_ctx* ctx, double* out, int32_t mem)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    if (ctx->P > 0 && !out) return fail(SIM_EINVAL, "null output");
    if (mem != SIM_MEM_HOST && mem != SIM_MEM_DEVICE) return fail(SIM_EINVAL, "bad mem %d", mem);
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    double* dst = mem == SIM_MEM_DEVICE ? out : ctx->d_fit.p;
    VX_LAUNCH(ctx, launch_fitness(ctx->view(), ctx->d_mass_corner.p, ctx->d_x.p, ctx->d_x0.p,
                                  (float)ctx->p.dead_bound, dst, s));
    if (mem == SIM_MEM_HOST) {
        // the status words ride along: a segmented lattice step that gave up waiting shows here
        int32_t words[4];
        VX_CK(cudaMemcpyAsync(words, ctx->d_status.p, sizeof(words), cudaMemcpyDeviceToHost, s));
        if (sim_status st = copy_out(out, ctx->d_fit.p, sizeof(double) * ctx->P, mem, s)) return st;
        const int32_t step_words[4] = {0, 0, words[2], 0};   // the population's own were reported
        return status_from_words(step_words);
    }
    return SIM_OK;
}

sim_status evo_generation(voxsim_ctx* ctx, const double* fitness, const float* genomes_in,
                          float* genomes_out, int32_t P, int32_t G, const evo_params* e,
                          uint64_t generation, int32_t* parents_out, uint8_t* mask_out)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!e || !fitness || !genomes_out) return fail(SIM_EINVAL, "null argument");
    if (!genomes_in) {       // the genome rows the last sim_set_population copied from the host
        if (ctx->host_genome_floats == 0)
            return fail(SIM_ESTATE, "genomes_in is NULL but the population was not set from host genome rows");
        if ((int64_t)P * G != ctx->host_genome_floats)
            return fail(SIM_EINVAL, "P x G = %lld does not match the %lld floats of the population's genome rows",
                        (long long)P * G, (long long)ctx->host_genome_floats);
        genomes_in = ctx->d_in_f32.p;
    }
    if (P < 1 || P > 65535) return fail(SIM_EINVAL, "P must be in 1..65535");
    if (G < 1 || G > (1 << 26)) return fail(SIM_EINVAL, "G must be in 1..2^26");
    if (e->elites < 1 || e->elites > P) return fail(SIM_EINVAL, "elites must be in 1..P");
    if (generation >= (1ull << 19)) return fail(SIM_EINVAL, "generation must be < 2^19");
    if (!(e->sigma >= 0.f)) return fail(SIM_EINVAL, "sigma must be >= 0");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    VX_CK(ctx->d_order.ensure(P));
    const float* src = genomes_in;
    const size_t n = (size_t)P * G;
    const float* lo_in = genomes_in; const float* hi_in = genomes_in + n;
    const float* lo_out = genomes_out; const float* hi_out = genomes_out + n;
    if (lo_in < hi_out && lo_out < hi_in) {   // overlapping: read from a copy
        VX_CK(ctx->d_gcopy.ensure(n));
        VX_CK(cudaMemcpyAsync(ctx->d_gcopy.p, genomes_in, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        src = ctx->d_gcopy.p;
    }
    VX_LAUNCH(ctx, launch_evo_rank(fitness, P, ctx->d_order.p, s));
    VX_LAUNCH(ctx, launch_evo_children(src, genomes_out, ctx->d_order.p, P, G, e->elites, e->seed, generation,
                              e->mut_threshold, e->sigma, e->keep_threshold, parents_out, mask_out, s));
    return SIM_OK;
}

sim_status evo_elite_weights(voxsim_ctx* ctx, const double* fitness, int32_t P, int32_t E, double* weights)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!fitness || !weights) return fail(SIM_EINVAL, "null argument");
    if (P < 1 || P > 65535) return fail(SIM_EINVAL, "P must be in 1..65535");
    if (E < 0 || E > P) return fail(SIM_EINVAL, "E must be in 0..P");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    VX_CK(ctx->d_order.ensure(P));
    VX_LAUNCH(ctx, launch_evo_rank(fitness, P, ctx->d_order.p, s));
    VX_LAUNCH(ctx, launch_elite_weights(ctx->d_order.p, fitness, P, E, weights, s));
    return SIM_OK;
}

// Lamarckian gradient step on genome rows [w | kappa | phi] of the current population.
sim_status evo_gradient_step(voxsim_ctx* ctx, float* genomes, int32_t P, int32_t G, const float* g_w,
                             const float* g_kappa, const float* g_phi, const int32_t* rows,
                             int32_t n_rows, float eta_w, float eta_kappa, float eta_phi,
                             const float* lo, const float* hi)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    if (P != ctx->P || P < 1) return fail(SIM_EINVAL, "P must equal the population size %d", ctx->P);
    for (int r = 1; r < P; ++r)
        if (ctx->dims[3 * r] != ctx->dims[0] || ctx->dims[3 * r + 1] != ctx->dims[1] || ctx->dims[3 * r + 2] != ctx->dims[2])
            return fail(SIM_EINVAL, "the gradient step needs one grid shape for all robots");
    const int64_t V = (int64_t)ctx->dims[0] * ctx->dims[1] * ctx->dims[2];
    if ((int64_t)G != 3 * V) return fail(SIM_EINVAL, "G must be 3 x voxels per robot = %lld", (long long)(3 * V));
    if (!genomes || !g_w || !g_kappa || !g_phi) return fail(SIM_EINVAL, "null genomes or gradients");
    if (!std::isfinite(eta_w) || !std::isfinite(eta_kappa) || !std::isfinite(eta_phi))
        return fail(SIM_EINVAL, "step sizes must be finite");
    std::vector<int> list;
    if (rows) {
        if (n_rows < 0 || n_rows > P) return fail(SIM_EINVAL, "n_rows must be in 0..P");
        for (int i = 0; i < n_rows; ++i) {
            if (rows[i] < 0 || rows[i] >= P) return fail(SIM_EINVAL, "row %d out of range", rows[i]);
            list.push_back(rows[i]);
        }
    } else {
        for (int r = 0; r < P; ++r) list.push_back(r);
    }
    if (list.empty()) return SIM_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    VX_CK(ctx->d_grad_rows.ensure(list.size()));
    VX_CK(cudaMemcpyAsync(ctx->d_grad_rows.p, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, s));
    VX_LAUNCH(ctx, launch_grad_step(genomes, G, V, ctx->d_voff.p, g_w, g_kappa, g_phi, ctx->d_grad_rows.p,
                                    (int)list.size(), eta_w, eta_kappa, eta_phi, lo, hi, s));
    // the row list is copied from pageable memory
    VX_CK(cudaStreamSynchronize(s));
    return SIM_OK;
}

sim_status sim_set_checkpointing(voxsim_ctx* ctx, int32_t k_steps)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (k_steps < 0) return fail(SIM_EINVAL, "k_steps must be >= 0");
    if (k_steps > 0 && ctx->p.accumulate == SIM_ACC_ATOMIC)
        return fail(SIM_EINVAL, "checkpointing needs the bit-reproducible stepping (not SIM_ACC_ATOMIC)");
    if (k_steps > 0 && (ctx->p.spring_zeta != 0.0 || ctx->p.ground_zeta != 0.0))
        return fail(SIM_EINVAL, "the adjoint is built for undamped springs and ground (zeta = 0)");
    const bool changed = (ctx->ckpt_every > 0) != (k_steps > 0);
    ctx->ckpt_every = k_steps;
    ctx->rec_valid = false;
    ctx->drop_graph();
    if (changed && ctx->have_pop && ctx->P > 0) {   // robots on the atomic kernel move to (or back from) the streamed path
        DeviceGuard g(ctx->device);
        if (sim_status st = build_work_items(ctx)) return st;
    }
    return SIM_OK;
}

sim_status sim_set_trajectory_records(voxsim_ctx* ctx, int32_t on)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (on != 0 && on != 1) return fail(SIM_EINVAL, "on must be 0 or 1");
    ctx->keep_records = on != 0;
    ctx->rec_valid = false;
    ctx->rec_full = false;
    if (!on) {
        DeviceGuard g(ctx->device);
        ctx->d_trec_u.release();
        ctx->d_trec_f.release();
    }
    return SIM_OK;
}

// The adjoint of the robots on the lattice kernels: per checkpoint segment, last to first, the
// forward per-corner lattice kernel replays the segment from a copy of its checkpoint in
// recording mode, then the reverse-sweep kernel runs over the records; adjoints and sensitivity
// sums are carried between segments in device memory.  When the forward kept every step's
// record, one reverse sweep runs over the whole run and nothing is replayed.  The checkpoints
// and records stay intact, so the backward pass may be repeated (other dL_df) on the same
// recorded run.
static sim_status backward_lattice(voxsim_ctx* ctx, const double* dL_df)
{
    cudaStream_t s = ctx->stream;
    const bool full = ctx->records_usable();
    const int N = ctx->rec_n, K = full ? N : ctx->ckpt_every;
    const size_t Mc = ctx->M_cap;
    // Without every step's record the backward replays each checkpoint segment (last to first)
    // before its reverse sweep.  The replays run on a second stream into two record buffers, so
    // the replay of segment s - 1 overlaps the sweep of segment s (each a persistent launch whose
    // last wave leaves SMs idle): the sweep of s waits for its replay, and the replay into a
    // buffer waits for the sweep that read it before.
    cudaStream_t r = s;
    if (!full) {
        VX_CK(ctx->d_srec_u.ensure(2 * (size_t)K * Mc));
        VX_CK(ctx->d_srec_f.ensure(2 * (size_t)K * Mc));
        VX_CK(ctx->d_slu.ensure(Mc)); VX_CK(ctx->d_slv.ensure(Mc));
        VX_CK(ctx->d_sacc.ensure(39 * Mc));
        VX_CK(ctx->d_rep_u0.ensure(Mc)); VX_CK(ctx->d_rep_v0.ensure(Mc));
        VX_CK(ctx->d_rep_u1.ensure(Mc)); VX_CK(ctx->d_rep_v1.ensure(Mc));
        if (!ctx->replay_stream) VX_CK(cudaStreamCreateWithFlags(&ctx->replay_stream, cudaStreamNonBlocking));
        for (cudaEvent_t& e : ctx->ev_bwd)
            if (!e) VX_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        r = ctx->replay_stream;
        VX_CK(cudaEventRecord(ctx->ev_bwd[4], s));     // the forward run and the zeroed sums
        VX_CK(cudaStreamWaitEvent(r, ctx->ev_bwd[4], 0));
    }
    const int threads = lattice_max_threads();
    const size_t smem = sizeof(float4) * kLatticeSlotVec4 * (size_t)threads;
    const int grid = std::min(ctx->n_items, ctx->num_sms);
    LatticeArgs f{};
    f.pv = ctx->view();
    f.corner_order = ctx->d_mass_corner.p;
    f.cflags = ctx->d_cflags.p;
    f.prm = ctx->d_prm.p;
    f.c = ctx->stepconst();
    f.items = ctx->d_items.p;
    f.item_robots = ctx->d_item_robots.p;
    f.n_items = ctx->n_items;
    f.cube8 = ctx->corner_cube8 && ctx->n_items == ctx->n_items_corner ? 1 : 0;
    f.queue = ctx->d_queue.p;
    f.rec_u = ctx->d_srec_u.p;
    f.rec_f = ctx->d_srec_f.p;
    f.rec_stride = (int64_t)Mc;
    ctx->imposed_args(f, ctx->rec_step0);
    AdjointArgs a{};
    a.pv = ctx->view();
    a.cflags = ctx->d_cflags.p;
    a.prm = ctx->d_prm.p;
    a.mat = ctx->d_mat.p;
    a.u0 = ctx->d_x.p;
    a.rec_u = full ? ctx->d_trec_u.p : ctx->d_srec_u.p;
    a.rec_f = full ? ctx->d_trec_f.p : ctx->d_srec_f.p;
    a.rec_stride = (int64_t)Mc;
    a.lu = ctx->d_slu.p;
    a.lv = ctx->d_slv.p;
    a.acc = ctx->d_sacc.p;
    a.sc = ctx->d_sc_rec.p;
    a.c = ctx->stepconst();
    a.dL_df = dL_df;
    a.items = ctx->d_items.p;
    a.item_robots = ctx->d_item_robots.p;
    a.n_items = ctx->n_items;
    a.cube8 = f.cube8;
    a.queue = ctx->d_queue.p;
    a.g_k = ctx->d_gk.p;
    a.g_a = ctx->d_ga.p;
    a.g_b = ctx->d_gb.p;
    const int nseg = (N + K - 1) / K;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int n0 = seg * K, n1 = std::min(N, n0 + K);
        if (!full) {
            const int b = seg & 1;                     // record buffer of this segment
            if (seg + 2 <= nseg - 1) VX_CK(cudaStreamWaitEvent(r, ctx->ev_bwd[2 + b], 0));
            float4* u0 = b ? ctx->d_rep_u1.p : ctx->d_rep_u0.p;
            float4* v0 = b ? ctx->d_rep_v1.p : ctx->d_rep_v0.p;
            VX_CK(cudaMemcpyAsync(u0, ctx->d_ckpt_u.p + (size_t)seg * Mc, sizeof(float4) * Mc,
                                  cudaMemcpyDeviceToDevice, r));
            VX_CK(cudaMemcpyAsync(v0, ctx->d_ckpt_v.p + (size_t)seg * Mc, sizeof(float4) * Mc,
                                  cudaMemcpyDeviceToDevice, r));
            f.u = u0;
            f.v = v0;
            f.rec_u = ctx->d_srec_u.p + (size_t)b * K * Mc;
            f.rec_f = ctx->d_srec_f.p + (size_t)b * K * Mc;
            f.sc = ctx->d_sc_rec.p + n0;
            f.nsteps = n1 - n0;
            f.imp_step0 = ctx->rec_step0 + n0;
            f.queue = ctx->d_queue.p + 1;
            VX_CK(cudaMemsetAsync(f.queue, 0, sizeof(int), r));
            VX_LAUNCH(ctx, launch_step_lattice(f, grid, threads, smem, r));
            VX_CK(cudaEventRecord(ctx->ev_bwd[b], r));
            VX_CK(cudaStreamWaitEvent(s, ctx->ev_bwd[b], 0));
            a.rec_u = f.rec_u;
            a.rec_f = f.rec_f;
        }
        a.n0 = n0;
        a.n1 = n1;
        a.first = seg == nseg - 1;
        a.last = seg == 0;
        VX_CK(cudaMemsetAsync(ctx->d_queue.p, 0, sizeof(int), s));
        // slots plus the double-buffered record staging (a float4 and a float2 per thread)
        VX_LAUNCH(ctx, launch_adjoint_lattice(a, grid, threads, smem + (size_t)threads * 2 * (16 + 8), s));
        if (!full) VX_CK(cudaEventRecord(ctx->ev_bwd[2 + (seg & 1)], s));   // its record buffer is free
    }
    return SIM_OK;
}

// The adjoint of the streamed robots: per checkpoint segment, last to first, a recording replay
// (the streamed step kernel) and a reverse sweep of one launch per step; the per-voxel
// sensitivity sums go to the same accumulators as the resident adjoint's.
static sim_status backward_streamed(voxsim_ctx* ctx, const double* dL_df)
{
    cudaStream_t s = ctx->stream;
    const bool full = ctx->records_usable();      // every step's record kept: no replay
    const int N = ctx->rec_n, K = full ? N : ctx->ckpt_every;
    const size_t Mc = ctx->M_cap;
    if (!full) {
        VX_CK(ctx->d_srec_u.ensure((size_t)K * Mc));
        VX_CK(ctx->d_srec_f.ensure((size_t)K * Mc));
        VX_CK(ctx->d_rep_u0.ensure(Mc)); VX_CK(ctx->d_rep_u1.ensure(Mc));
        VX_CK(ctx->d_rep_v0.ensure(Mc)); VX_CK(ctx->d_rep_v1.ensure(Mc));
    }
    float4* const rec_u = full ? ctx->d_trec_u.p : ctx->d_srec_u.p;
    float2* const rec_f = full ? ctx->d_trec_f.p : ctx->d_srec_f.p;
    VX_CK(ctx->d_slu.ensure(Mc)); VX_CK(ctx->d_slv.ensure(Mc));
    VX_CK(ctx->d_slF0.ensure(Mc)); VX_CK(ctx->d_slF1.ensure(Mc));
    VX_CK(ctx->d_sacc.ensure(39 * Mc));
    StreamAdjArgs b{};
    b.pv = ctx->view();
    b.cflags = ctx->d_cflags.p;
    b.prm = ctx->d_prm.p;
    b.mat = ctx->d_mat.p;
    b.u0 = ctx->d_x.p;
    b.lu = ctx->d_slu.p;
    b.lv = ctx->d_slv.p;
    b.acc = ctx->d_sacc.p;
    b.sc = ctx->d_sc_rec.p;
    b.dL_df = dL_df;
    b.c = ctx->stepconst();
    b.robots = ctx->d_stream.p;
    b.cube40 = ctx->stream_cube40 ? 1 : 0;
    b.n_robots = ctx->n_stream;
    b.g_k = ctx->d_gk.p;
    b.g_a = ctx->d_ga.p;
    b.g_b = ctx->d_gb.p;
    const int maxc = ctx->max_stream_corner;
    VX_LAUNCH(ctx, launch_stream_adj_init(b, maxc, s));
    float4* lF[2] = {ctx->d_slF0.p, ctx->d_slF1.p};
    float4* ru[2] = {ctx->d_rep_u0.p, ctx->d_rep_u1.p};
    float4* rv[2] = {ctx->d_rep_v0.p, ctx->d_rep_v1.p};
    StreamArgs f{};
    f.pv = ctx->view();
    f.cflags = ctx->d_cflags.p;
    f.prm = ctx->d_prm.p;
    f.sc = ctx->d_sc_rec.p;
    f.c = ctx->stepconst();
    f.robots = ctx->d_stream.p;
    f.n_robots = ctx->n_stream;
    f.cube40 = ctx->stream_cube40 ? 1 : 0;
    const int nseg = (N + K - 1) / K;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int n0 = seg * K, n1 = std::min(N, n0 + K);
        // replay from the checkpoint, recording every step
        for (int i = 0; i < n1 - n0 && !full; ++i) {
            f.u_in = i == 0 ? ctx->d_ckpt_u.p + (size_t)seg * Mc : ru[(i - 1) & 1];
            f.v_in = i == 0 ? ctx->d_ckpt_v.p + (size_t)seg * Mc : rv[(i - 1) & 1];
            f.u_out = ru[i & 1];
            f.v_out = rv[i & 1];
            f.rec_u = ctx->d_srec_u.p + (size_t)i * Mc;
            f.rec_f = ctx->d_srec_f.p + (size_t)i * Mc;
            VX_LAUNCH(ctx, launch_step_streamed(f, n0 + i, maxc, s));
        }
        // the mass part of the segment's last step, then per step its spring part and the mass
        // part of the step before it
        for (int j = n1; j >= n0; --j) {
            b.step = j < n1 ? j : -1;
            b.rec_u = j < n1 ? rec_u + (size_t)(j - n0) * Mc : nullptr;
            b.lF_in = j < n1 ? lF[j & 1] : nullptr;
            const bool mass = j - 1 >= n0;
            b.mrec_u = mass ? rec_u + (size_t)(j - 1 - n0) * Mc : nullptr;
            b.mrec_f = mass ? rec_f + (size_t)(j - 1 - n0) * Mc : nullptr;
            b.lF_out = mass ? lF[(j - 1) & 1] : nullptr;
            VX_LAUNCH(ctx, launch_stream_adj_step(b, maxc, s));
        }
    }
    VX_LAUNCH(ctx, launch_stream_adj_voxels(b, maxc, s));
    return SIM_OK;
}

// Contact modes of one robot over the recorded run: the checkpoint segments are replayed in
// recording mode (lattice robots with the per-corner kernel, streamed robots with the streamed
// kernel, both as in sim_backward) and the robot's mode field copied out segment by segment.
sim_status sim_get_contact_modes(voxsim_ctx* ctx, int32_t robot, uint8_t* out)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop || !ctx->rec_valid) return fail(SIM_ESTATE, "no recorded forward run");
    if (robot < 0 || robot >= ctx->P) return fail(SIM_EINVAL, "robot %d out of range", robot);
    if (!out) return fail(SIM_EINVAL, "null output");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const int K = ctx->ckpt_every, N = ctx->rec_n;
    const size_t Mc = ctx->M_cap;
    const int r = robot;
    const int C = (ctx->dims[3 * r] + 1) * (ctx->dims[3 * r + 1] + 1) * (ctx->dims[3 * r + 2] + 1);
    const int64_t mo = ctx->moff[r];
    bool streamed = false;
    for (int q : ctx->stream_robots) streamed = streamed || q == r;
    VX_CK(ctx->d_sc_rec.ensure(N));
    VX_LAUNCH(ctx, launch_sincos_table(2.0 * 3.141592653589793 * ctx->p.freq, ctx->p.dt, ctx->rec_step0, N,
                                       ctx->d_sc_rec.p, s));
    VX_CK(ctx->d_srec_u.ensure((size_t)K * Mc));
    VX_CK(ctx->d_srec_f.ensure((size_t)K * Mc));
    VX_CK(ctx->d_rep_u0.ensure(Mc)); VX_CK(ctx->d_rep_v0.ensure(Mc));
    VX_CK(ctx->d_rep_u1.ensure(Mc)); VX_CK(ctx->d_rep_v1.ensure(Mc));
    std::vector<uint32_t> fl(C);
    VX_CK(cudaMemcpyAsync(fl.data(), ctx->d_cflags.p + mo, sizeof(uint32_t) * C, cudaMemcpyDeviceToHost, s));
    std::vector<float4> rec((size_t)K * C);
    const int nseg = (N + K - 1) / K;
    for (int seg = 0; seg < nseg; ++seg) {
        const int n0 = seg * K, n1 = std::min(N, n0 + K);
        const float4* src = ctx->d_srec_u.p;
        if (ctx->records_usable()) {           // the forward kept every step's record
            src = ctx->d_trec_u.p + (size_t)n0 * Mc;
        } else if (!streamed) {
            LatticeArgs f{};
            f.pv = ctx->view();
            f.corner_order = ctx->d_mass_corner.p;
            f.cflags = ctx->d_cflags.p;
            f.prm = ctx->d_prm.p;
            f.c = ctx->stepconst();
            f.items = ctx->d_items.p;
            f.item_robots = ctx->d_item_robots.p;
            f.n_items = ctx->n_items;
            f.cube8 = ctx->corner_cube8 && ctx->n_items == ctx->n_items_corner ? 1 : 0;
            f.queue = ctx->d_queue.p;
            f.rec_u = ctx->d_srec_u.p;
            f.rec_f = ctx->d_srec_f.p;
            f.rec_stride = (int64_t)Mc;
            VX_CK(cudaMemcpyAsync(ctx->d_rep_u0.p, ctx->d_ckpt_u.p + (size_t)seg * Mc, sizeof(float4) * Mc,
                                  cudaMemcpyDeviceToDevice, s));
            VX_CK(cudaMemcpyAsync(ctx->d_rep_v0.p, ctx->d_ckpt_v.p + (size_t)seg * Mc, sizeof(float4) * Mc,
                                  cudaMemcpyDeviceToDevice, s));
            f.u = ctx->d_rep_u0.p;
            f.v = ctx->d_rep_v0.p;
            f.sc = ctx->d_sc_rec.p + n0;
            f.nsteps = n1 - n0;
            ctx->imposed_args(f, ctx->rec_step0 + n0);
            const int threads = lattice_max_threads();
            VX_CK(cudaMemsetAsync(ctx->d_queue.p, 0, sizeof(int), s));
            VX_LAUNCH(ctx, launch_step_lattice(f, std::min(ctx->n_items, ctx->num_sms), threads,
                                               sizeof(float4) * kLatticeSlotVec4 * (size_t)threads, s));
        } else {
            StreamArgs f{};
            f.pv = ctx->view();
            f.cflags = ctx->d_cflags.p;
            f.prm = ctx->d_prm.p;
            f.sc = ctx->d_sc_rec.p;
            f.c = ctx->stepconst();
            f.robots = ctx->d_stream.p;
            f.n_robots = ctx->n_stream;
            f.cube40 = ctx->stream_cube40 ? 1 : 0;
            float4* ru[2] = {ctx->d_rep_u0.p, ctx->d_rep_u1.p};
            float4* rv[2] = {ctx->d_rep_v0.p, ctx->d_rep_v1.p};
            for (int i = 0; i < n1 - n0; ++i) {
                f.u_in = i == 0 ? ctx->d_ckpt_u.p + (size_t)seg * Mc : ru[(i - 1) & 1];
                f.v_in = i == 0 ? ctx->d_ckpt_v.p + (size_t)seg * Mc : rv[(i - 1) & 1];
                f.u_out = ru[i & 1];
                f.v_out = rv[i & 1];
                f.rec_u = ctx->d_srec_u.p + (size_t)i * Mc;
                f.rec_f = ctx->d_srec_f.p + (size_t)i * Mc;
                VX_LAUNCH(ctx, launch_step_streamed(f, n0 + i, ctx->max_stream_corner, s));
            }
        }
        VX_CK(cudaMemcpy2DAsync(rec.data(), sizeof(float4) * C, src + mo, sizeof(float4) * Mc,
                                sizeof(float4) * C, n1 - n0, cudaMemcpyDeviceToHost, s));
        VX_CK(cudaStreamSynchronize(s));
        for (int j = 0; j < n1 - n0; ++j)
            for (int c = 0; c < C; ++c) {
                uint32_t mode = 0u;
                if (fl[c] >> 31) std::memcpy(&mode, &rec[(size_t)j * C + c].w, sizeof(mode));
                out[(size_t)(n0 + j) * C + c] = (uint8_t)mode;
            }
    }
    return SIM_OK;
}

sim_status sim_backward(voxsim_ctx* ctx, const double* dL_df, float* g_w, float* g_kappa, float* g_phi)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop || !ctx->rec_valid) return fail(SIM_ESTATE, "no recorded forward run");
    if (ctx->P > 0 && (!dL_df || !g_w || !g_kappa || !g_phi)) return fail(SIM_EINVAL, "null argument");
    if (ctx->P == 0 || ctx->rec_n == 0) return SIM_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const size_t V = ctx->V_tot;
    VX_CK(ctx->d_gk.ensure(V)); VX_CK(ctx->d_ga.ensure(V)); VX_CK(ctx->d_gb.ensure(V));
    VX_CK(cudaMemsetAsync(ctx->d_gk.p, 0, sizeof(float) * V, s));
    VX_CK(cudaMemsetAsync(ctx->d_ga.p, 0, sizeof(float) * V, s));
    VX_CK(cudaMemsetAsync(ctx->d_gb.p, 0, sizeof(float) * V, s));
    VX_CK(ctx->d_sc_rec.ensure(ctx->rec_n));
    VX_LAUNCH(ctx, launch_sincos_table(2.0 * 3.141592653589793 * ctx->p.freq, ctx->p.dt, ctx->rec_step0,
                                       ctx->rec_n, ctx->d_sc_rec.p, s));
    if (ctx->n_items > 0)
        if (sim_status st = backward_lattice(ctx, dL_df)) return st;
    if (ctx->n_stream > 0)
        if (sim_status st = backward_streamed(ctx, dL_df)) return st;
    VX_LAUNCH(ctx, launch_adjoint_voxels(ctx->d_mat.p, ctx->d_w.p, ctx->d_kappa.p, ctx->d_phi.p, ctx->matconst(),
                                         ctx->d_gk.p, ctx->d_ga.p, ctx->d_gb.p, (int64_t)V, g_w, g_kappa, g_phi, s));
    return SIM_OK;
}

// Diversity of a population: genomes (optional, device [P][G]) and the current population's
// kept material grids (all robots on one grid shape).
sim_status sim_diversity(voxsim_ctx* ctx, const float* genomes, int32_t P, int32_t G, double* out)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!out) return fail(SIM_EINVAL, "null output");
    if (P < 2) return fail(SIM_EINVAL, "diversity needs at least two robots");
    if (genomes && G < 1) return fail(SIM_EINVAL, "G must be >= 1");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    bool morph = ctx->have_pop && ctx->P == P && P > 0;
    for (int r = 1; morph && r < P; ++r)
        morph = ctx->dims[3 * r] == ctx->dims[0] && ctx->dims[3 * r + 1] == ctx->dims[1] && ctx->dims[3 * r + 2] == ctx->dims[2];
    const int V = morph ? ctx->dims[0] * ctx->dims[1] * ctx->dims[2] : 0;
    VX_CK(ctx->d_fit.ensure(std::max(2, ctx->P)));
    VX_LAUNCH(ctx, launch_diversity(genomes, P, genomes ? G : 0, morph ? ctx->d_mat.p : nullptr, V, ctx->d_fit.p, s));
    double tot[2];
    if (sim_status st = copy_out(tot, ctx->d_fit.p, sizeof(tot), SIM_MEM_HOST, s)) return st;
    out[0] = genomes ? std::sqrt(2.0 * tot[0] / (P - 1.0)) : NAN;
    out[1] = morph ? tot[1] / (0.5 * P * (P - 1.0)) / V : NAN;
    return SIM_OK;
}

// Per size class, time every admissible kernel on a sample of the class's robots (up to two per
// SM) for n_steps steps from the current state, keep the fastest, restore the state.
sim_status sim_impose_contact_modes(voxsim_ctx* ctx, int32_t robot, const uint8_t* modes, int32_t n_steps)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    DeviceGuard g(ctx->device);
    if (!modes) {
        const bool was = ctx->imp_active;
        ctx->imp_active = false;
        ctx->imp_n = 0;
        ctx->imp_off.clear();
        ctx->imp_table.clear();
        ctx->rec_valid = false;
        if (was) return build_work_items(ctx);
        return SIM_OK;
    }
    if (robot < 0 || robot >= ctx->P) return fail(SIM_EINVAL, "robot %d out of range", robot);
    if (n_steps < 1) return fail(SIM_EINVAL, "n_steps must be >= 1");
    if (ctx->imp_active && n_steps != ctx->imp_n)
        return fail(SIM_EINVAL, "every imposed robot must cover the same %d steps", ctx->imp_n);
    if (ctx->stepconst().damped || ctx->p.ground_zeta != 0.0)
        return fail(SIM_EINVAL, "imposed contact modes need undamped springs and ground");
    if (ctx->p.path == SIM_PATH_STREAMED || ctx->p.path == SIM_PATH_PLAIN || ctx->p.accumulate == SIM_ACC_ATOMIC)
        return fail(SIM_EINVAL, "imposed contact modes run on the lattice kernel");
    const int C = (ctx->dims[3 * robot] + 1) * (ctx->dims[3 * robot + 1] + 1) * (ctx->dims[3 * robot + 2] + 1);
    if (C > lattice_max_threads())
        return fail(SIM_EINVAL, "robot %d (%d corners) is not on the lattice kernel", robot, C);
    const size_t len = (size_t)n_steps * C;
    for (size_t i = 0; i < len; ++i)
        if (modes[i] > 3) return fail(SIM_EINVAL, "contact mode %d out of range 0..3", (int)modes[i]);
    if (ctx->imp_off.size() != (size_t)ctx->P) ctx->imp_off.assign(ctx->P, -1);
    int64_t off = ctx->imp_off[robot];
    if (off < 0) {
        off = (int64_t)ctx->imp_table.size();
        ctx->imp_table.resize(ctx->imp_table.size() + len);
        ctx->imp_off[robot] = off;
    }
    std::memcpy(ctx->imp_table.data() + off, modes, len);
    VX_CK(ctx->d_imp_modes.ensure(ctx->imp_table.size()));
    VX_CK(ctx->d_imp_off.ensure(ctx->P));
    cudaStream_t s = ctx->stream;
    VX_CK(cudaMemcpyAsync(ctx->d_imp_modes.p, ctx->imp_table.data(), ctx->imp_table.size(), cudaMemcpyHostToDevice, s));
    VX_CK(cudaMemcpyAsync(ctx->d_imp_off.p, ctx->imp_off.data(), sizeof(int64_t) * ctx->P, cudaMemcpyHostToDevice, s));
    VX_CK(cudaStreamSynchronize(s));
    const bool was = ctx->imp_active;
    ctx->imp_active = true;
    ctx->imp_n = n_steps;
    ctx->rec_valid = false;
    if (!was) return build_work_items(ctx);      // per-corner kernel only while modes are imposed
    return SIM_OK;
}

sim_status sim_autotune(voxsim_ctx* ctx, int32_t n_steps, int32_t* kind_out, int32_t* threads_out)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    if (n_steps < 1) return fail(SIM_EINVAL, "n_steps must be >= 1");
    if (ctx->p.path == SIM_PATH_PLAIN) return fail(SIM_EINVAL, "the plain path has nothing to tune");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const size_t Mc = ctx->M_cap;
    DevBuf<float4> snap_u, snap_v;
    VX_CK(snap_u.ensure(Mc));
    VX_CK(snap_v.ensure(Mc));
    VX_CK(cudaMemcpyAsync(snap_u.p, ctx->d_x.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
    VX_CK(cudaMemcpyAsync(snap_v.p, ctx->d_v.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
    VX_CK(ctx->d_sc.ensure(n_steps));
    VX_LAUNCH(ctx, launch_sincos_table(2.0 * 3.141592653589793 * ctx->p.freq, ctx->p.dt, ctx->step, n_steps,
                                       ctx->d_sc.p, s));
    if (!ctx->tuned) default_choices(ctx);
    ctx->tuned = true;
    std::vector<std::vector<std::pair<int, int>>> members(kNumClasses);
    for (int r = 0; r < ctx->P; ++r) {
        const int C = (ctx->dims[3 * r] + 1) * (ctx->dims[3 * r + 1] + 1) * (ctx->dims[3 * r + 2] + 1);
        members[class_of(C)].push_back({-C, r});
    }
    const size_t budget = ctx->smem_optin > 2048 ? ctx->smem_optin - 1024 : ctx->smem_optin;
    cudaEvent_t e0, e1;
    VX_CK(cudaEventCreate(&e0));
    VX_CK(cudaEventCreate(&e1));
    sim_status result = SIM_OK;
    for (int k = 0; k < kNumClasses && result == SIM_OK; ++k) {
        if (members[k].empty()) continue;
        std::sort(members[k].begin(), members[k].end());
        std::vector<int> sample;
        // up to six robots per SM of the class: enough waves that the tail of a launch, which a
        // candidate splitting the class over two launches pays twice, does not decide the choice
        for (size_t i = 0; i < members[k].size() && (int)i < 6 * ctx->num_sms; ++i) sample.push_back(members[k][i].second);
        const int Cmax = -members[k].front().first;
        const bool fits = Cmax <= kResidentMaxCorner && resident_smem_bytes(Cmax, 0, SIM_ACC_ATOMIC) <= budget;
        std::vector<std::pair<int, int>> cands;
        if (k < 6 && ctx->p.accumulate != SIM_ACC_ATOMIC) {
            if (ctx->p.lattice != SIM_LATTICE_COMPACT) cands.push_back({kKindLattice, 0});
            if (ctx->p.lattice != SIM_LATTICE_CORNER && ctx->p.lattice != SIM_LATTICE_PACKED && ctx->have_pack)
                cands.push_back({kKindLatticeCompact, 0});
        }
        if (fits && ctx->p.accumulate != SIM_ACC_GATHER) {
            const int t3[3] = {k < 6 ? 128 : 256, k < 6 ? 256 : 512, k < 6 ? 512 : 1024};
            for (int t : t3) cands.push_back({kKindAtomic, t});
        }
        if (k >= 6 && ctx->p.path != SIM_PATH_STREAMED && cluster_q(ctx->dims[3 * sample[0]], ctx->dims[3 * sample[0] + 1],
                                                                   ctx->dims[3 * sample[0] + 2]) >= 2)
            cands.push_back({kKindCluster, 0});
        if (k >= 6 && k < kNumClasses - 1 && ctx->p.accumulate != SIM_ACC_ATOMIC && ctx->ckpt_every == 0 &&
            ctx->p.path != SIM_PATH_STREAMED)
            cands.push_back({kKindMassGroups, 0});
        if (k >= 6 && ctx->p.path != SIM_PATH_RESIDENT) cands.push_back({kKindStreamed, 0});
        if (cands.size() < 2) continue;
        float best_ms = 1e30f;
        std::pair<int, int> best = cands.front();
        for (const auto& cand : cands) {
            ctx->class_kind[k] = cand.first;
            ctx->class_threads[k] = cand.second;
            if ((result = build_work_items(ctx, &sample)) != SIM_OK) break;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && result == SIM_OK; ++rep) {    // warm-up run, timed run
                VX_CK(cudaMemcpyAsync(ctx->d_x.p, snap_u.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
                VX_CK(cudaMemcpyAsync(ctx->d_v.p, snap_v.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
                if (ctx->n_stream > 0) {
                    VX_CK(cudaMemcpyAsync(ctx->d_x_alt.p, snap_u.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
                    VX_CK(cudaMemcpyAsync(ctx->d_v_alt.p, snap_v.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
                }
                VX_CK(cudaEventRecord(e0, s));
                if ((result = step_lattice(ctx, n_steps, false)) != SIM_OK) break;
                if ((result = step_cluster(ctx, n_steps)) != SIM_OK) break;
                if ((result = step_resident(ctx, n_steps)) != SIM_OK) break;
                if ((result = step_streamed(ctx, n_steps, false)) != SIM_OK) break;
                VX_CK(cudaEventRecord(e1, s));
                VX_CK(cudaEventSynchronize(e1));
                VX_CK(cudaEventElapsedTime(&ms, e0, e1));
            }
            if (result == SIM_OK && ms < best_ms) { best_ms = ms; best = cand; }
        }
        ctx->class_kind[k] = best.first;
        ctx->class_threads[k] = best.second;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    VX_CK(cudaMemcpyAsync(ctx->d_x.p, snap_u.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
    VX_CK(cudaMemcpyAsync(ctx->d_v.p, snap_v.p, sizeof(float4) * Mc, cudaMemcpyDeviceToDevice, s));
    if (result == SIM_OK) result = build_work_items(ctx);   // also resets the alternate buffer
    VX_CK(cudaStreamSynchronize(s));
    if (result != SIM_OK) return result;
    for (int k = 0; k < kNumClasses; ++k) {
        if (kind_out) kind_out[k] = ctx->class_kind[k];
        if (threads_out) threads_out[k] = ctx->class_threads[k];
    }
    return SIM_OK;
}

sim_status sim_get_counts(voxsim_ctx* ctx, int32_t* n_masses, int32_t* n_springs)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    if (n_masses && ctx->P) VX_CK(cudaMemcpyAsync(n_masses, ctx->d_nm.p, 4 * ctx->P, cudaMemcpyDeviceToHost, s));
    if (n_springs && ctx->P) VX_CK(cudaMemcpyAsync(n_springs, ctx->d_ns.p, 4 * ctx->P, cudaMemcpyDeviceToHost, s));
    VX_CK(cudaStreamSynchronize(s));
    return SIM_OK;
}

sim_status sim_get_state(voxsim_ctx* ctx, float* x_out, float* v_out, int32_t* mass_offsets, int32_t mem)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    if (mem != SIM_MEM_HOST && mem != SIM_MEM_DEVICE) return fail(SIM_EINVAL, "bad mem %d", mem);
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const int P = ctx->P;
    std::vector<int32_t> nm(P);
    if (sim_status st = sim_get_counts(ctx, nm.data(), nullptr)) return st;
    std::vector<int64_t> off(P + 1, 0);
    for (int r = 0; r < P; ++r) off[r + 1] = off[r] + nm[r];
    if (mass_offsets)
        for (int r = 0; r <= P; ++r) mass_offsets[r] = (int32_t)off[r];
    const int64_t Mt = off[P];
    if (P == 0 || Mt == 0) return SIM_OK;
    VX_CK(cudaMemcpyAsync(ctx->d_tmp_off.p, off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s));
    VX_CK(ctx->d_compact.ensure(3 * (size_t)Mt));
    float* outs[2] = {x_out, v_out};
    const float4* srcs[2] = {ctx->d_x.p, ctx->d_v.p};
    const float4* adds[2] = {ctx->d_x0.p, nullptr};   // position = rest lattice + displacement
    for (int i = 0; i < 2; ++i) {
        if (!outs[i]) continue;
        float* dst = mem == SIM_MEM_DEVICE ? outs[i] : ctx->d_compact.p;
        VX_LAUNCH(ctx, launch_compact_state(ctx->view(), ctx->d_mass_corner.p, srcs[i], adds[i], dst,
                                            ctx->d_tmp_off.p, s));
        if (mem == SIM_MEM_HOST)
            if (sim_status st = copy_out(outs[i], ctx->d_compact.p, sizeof(float) * 3 * Mt, mem, s)) return st;
    }
    VX_CK(cudaStreamSynchronize(s));
    return SIM_OK;
}

sim_status sim_get_voxels(voxsim_ctx* ctx, uint8_t* mat_decoded, uint8_t* mat_kept, float* w,
                          float* kappa, float* phi)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const size_t V = ctx->V_tot;
    if (mat_decoded) if (sim_status st = copy_out(mat_decoded, ctx->d_mat_raw.p, V, SIM_MEM_HOST, s)) return st;
    if (mat_kept) if (sim_status st = copy_out(mat_kept, ctx->d_mat.p, V, SIM_MEM_HOST, s)) return st;
    if (w) if (sim_status st = copy_out(w, ctx->d_w.p, 4 * V, SIM_MEM_HOST, s)) return st;
    if (kappa) if (sim_status st = copy_out(kappa, ctx->d_kappa.p, 4 * V, SIM_MEM_HOST, s)) return st;
    if (phi) if (sim_status st = copy_out(phi, ctx->d_phi.p, 4 * V, SIM_MEM_HOST, s)) return st;
    return SIM_OK;
}

sim_status sim_get_topology(voxsim_ctx* ctx, int32_t* mass_corner, int32_t* spring_ab, float* spring_params)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!ctx->have_pop) return fail(SIM_ESTATE, "no population set");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const int P = ctx->P;
    std::vector<int32_t> nm(P), ns(P);
    if (sim_status st = sim_get_counts(ctx, nm.data(), ns.data())) return st;
    if (mass_corner) {
        std::vector<int32_t> all(ctx->M_cap);
        if (sim_status st = copy_out(all.data(), ctx->d_mass_corner.p, 4 * ctx->M_cap, SIM_MEM_HOST, s)) return st;
        int64_t o = 0;
        for (int r = 0; r < P; ++r) {
            std::memcpy(mass_corner + o, all.data() + ctx->moff[r], 4 * (size_t)nm[r]);
            o += nm[r];
        }
    }
    if (spring_ab || spring_params) {
        std::vector<int2> ab(ctx->S_cap);
        std::vector<float4> sp(ctx->S_cap);
        if (sim_status st = copy_out(ab.data(), ctx->d_sab.p, sizeof(int2) * ctx->S_cap, SIM_MEM_HOST, s)) return st;
        if (sim_status st = copy_out(sp.data(), ctx->d_sp.p, sizeof(float4) * ctx->S_cap, SIM_MEM_HOST, s)) return st;
        int64_t o = 0;
        for (int r = 0; r < P; ++r) {
            for (int i = 0; i < ns[r]; ++i) {
                const int2 q = ab[ctx->soff[r] + i];
                const float4 t = sp[ctx->soff[r] + i];
                if (spring_ab) { spring_ab[2 * (o + i)] = q.x; spring_ab[2 * (o + i) + 1] = q.y; }
                if (spring_params) {
                    float* dst = spring_params + 4 * (o + i);
                    dst[0] = t.x; dst[1] = t.y; dst[2] = t.z; dst[3] = t.w;
                }
            }
            o += ns[r];
        }
    }
    return SIM_OK;
}

sim_status sim_get_timing(voxsim_ctx* ctx, double* step_ms, int64_t* launches)
{
    if (sim_status st = check_ctx(ctx)) return st;
    DeviceGuard g(ctx->device);
    VX_CK(cudaStreamSynchronize(ctx->stream));
    double total = 0.0;
    for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
        float ms = 0.f;
        VX_CK(cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
        total += ms;
    }
    if (step_ms) *step_ms = total;
    if (launches) *launches = ctx->launches;
    ctx->ev_used = 0;
    ctx->launches = 0;
    return SIM_OK;
}

sim_status sim_measure_smem_bandwidth(voxsim_ctx* ctx, double* gbs)
{
    if (sim_status st = check_ctx(ctx)) return st;
    if (!gbs) return fail(SIM_EINVAL, "null output");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const int grid = 2 * ctx->num_sms;            // two 1024-thread blocks per SM
    const int iters = 4000;                       // about 5 ms at the nominal rate
    float* sink = nullptr;
    VX_CK(cudaMallocAsync((void**)&sink, sizeof(float) * grid, s));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = launch_probe_smem(grid, iters / 4, sink, s);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = launch_probe_smem(grid, iters, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ctx->launches += 2;
    cudaFreeAsync(sink, s);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(e, "shared-memory probe");
    if (!(ms > 0.f)) return fail(SIM_ECUDA, "shared-memory probe: no elapsed time");
    *gbs = (double)probe_smem_bytes_per_iter(grid) * iters / (ms * 1e-3) / 1e9;
    return SIM_OK;
}

}  // extern "C"
