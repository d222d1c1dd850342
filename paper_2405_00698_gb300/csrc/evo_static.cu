// Allocation-free variant of the evolution step, for callers that must not allocate device
// memory (see evo_generation_static in include/voxsim.h).
//
// The only scratch the step needs is the rank order of the population.  Here it lives in a
// file-scope device array of fixed size instead of a context buffer: every GPU that loads the
// library holds it until the process exits, and every call on a device shares it.  Host code
// cannot use the array's name as a device address (it is a host-side stand-in), so the device
// address is taken once per device with cudaGetSymbolAddress while that device is current.
#include <mutex>

#include "common.cuh"

namespace vx {
namespace {

constexpr int kStaticMaxRobots = 16384;                   // 64 KB of device memory per GPU
constexpr int kMaxDevices = 64;

}  // namespace
}  // namespace vx

// Rank-order scratch of the allocation-free evolution step (shared by every call on a device).
static __device__ __align__(256) int g_static_order[vx::kStaticMaxRobots];

namespace vx {
namespace {

std::mutex g_setup_mutex;
int* g_order_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t static_order_address(int device, int** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_order_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_order);
        if (e != cudaSuccess) return e;
        g_order_addr[device] = static_cast<int*>(p);
    }
    *out = g_order_addr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace vx

using namespace vx;

extern "C" sim_status evo_generation_static(const double* fitness, const float* genomes_in,
                                            float* genomes_out, int32_t P, int32_t G,
                                            const evo_params* e, uint64_t generation,
                                            int32_t* parents_out, uint8_t* mask_out,
                                            void* cuda_stream)
{
    if (!e || !fitness || !genomes_in || !genomes_out) return vx_fail(SIM_EINVAL, "null argument");
    if (P < 1 || P > kStaticMaxRobots)
        return vx_fail(SIM_EINVAL, "P must be in 1..%d for the allocation-free evolution step", kStaticMaxRobots);
    if (G < 1 || G > (1 << 26)) return vx_fail(SIM_EINVAL, "G must be in 1..2^26");
    if (e->elites < 1 || e->elites > P) return vx_fail(SIM_EINVAL, "elites must be in 1..P");
    if (generation >= (1ull << 19)) return vx_fail(SIM_EINVAL, "generation must be < 2^19");
    if (!(e->sigma >= 0.f)) return vx_fail(SIM_EINVAL, "sigma must be >= 0");
    const size_t n = (size_t)P * G;
    if (genomes_in < genomes_out + n && genomes_out < genomes_in + n)
        return vx_fail(SIM_EINVAL, "genomes_in and genomes_out overlap (no scratch to copy into)");
    int device = 0;
    cudaError_t err = cudaGetDevice(&device);
    if (err != cudaSuccess) return vx_fail(SIM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(err));
    if (device < 0 || device >= kMaxDevices) return vx_fail(SIM_EINVAL, "device %d not supported", device);
    int* order = nullptr;
    err = static_order_address(device, &order);
    if (err != cudaSuccess) return vx_fail(SIM_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(err));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // every entry of the order array is written by the rank kernel, so nothing needs clearing
    err = launch_evo_rank(fitness, P, order, s);
    if (err != cudaSuccess) return vx_fail(SIM_ECUDA, "rank kernel: %s", cudaGetErrorString(err));
    err = launch_evo_children(genomes_in, genomes_out, order, P, G, e->elites, e->seed, generation,
                              e->mut_threshold, e->sigma, e->keep_threshold, parents_out, mask_out, s);
    if (err != cudaSuccess) return vx_fail(SIM_ECUDA, "crossover kernel: %s", cudaGetErrorString(err));
    return SIM_OK;
}
