// noalloc.cu - a kinetic-energy reduction that allocates no device memory.
//
// Some callers cannot allocate device memory when they need this value: hosts that
// hand this library a fixed memory budget and lock allocation after start-up (an
// embedding runtime that owns every byte of device memory through its own pool), and
// real-time loops that must not call cudaMalloc, which can synchronise the device and
// stall the loop.  md_kinetic_energy_noalloc serves them: it
// computes 1/2 sum m v^2 of caller-owned velocities with the same deterministic
// two-pass FP64 reduction as md_energy_virial, but keeps its per-CTA partial
// sums in one statically sized device array instead of allocating scratch.
#include "mdgb.h"
#include "mdgb_internal.cuh"

#include <mutex>

namespace {

constexpr int NOALLOC_MAX_PARTS = 1024;       // partial sums the static array holds
constexpr int NOALLOC_THREADS = 256;
constexpr long long NOALLOC_MAX_ATOMS = 1LL << 30;

// Scratch for the partial sums.  In host code this name is only a stand-in for the
// device symbol, never a device address: the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_PARTS];

struct NoallocMass {
    double m[mdgb::MAX_SPECIES];
};

// A species id outside [0, nsp) reads no mass: its term is NaN, so the sum reports it.
__global__ void __launch_bounds__(NOALLOC_THREADS) k_ke_partials(long long n, const double* __restrict__ vel,
                                                                  const int32_t* __restrict__ species, int nsp,
                                                                  NoallocMass mass, long long chunk,
                                                                  double* __restrict__ partials) {
    __shared__ double sh[NOALLOC_THREADS];
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += NOALLOC_THREADS) {
        const int a = species ? species[i] : 0;
        const double m = (a >= 0 && a < nsp) ? mass.m[a] : __longlong_as_double(0x7ff8000000000000LL);
        const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        acc += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = NOALLOC_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(NOALLOC_THREADS) k_ke_final(const double* __restrict__ partials, int nparts,
                                                              double* __restrict__ out) {
    __shared__ double sh[NOALLOC_THREADS];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nparts; b += NOALLOC_THREADS) acc += partials[b];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = NOALLOC_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Device address of the static array, looked up once per device with that device
// current (kept per device: every GPU that loads the library has its own copy).
constexpr int MAX_DEVICES = 64;
double* g_partials_addr[MAX_DEVICES] = {};
std::mutex g_partials_mutex;

int partials_for_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_partials_mutex);
    if (!g_partials_addr[dev]) {
        double* p = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_partials) != cudaSuccess || !p)
            return MD_ERR_CUDA;
        g_partials_addr[dev] = p;
    }
    *out = g_partials_addr[dev];
    return MD_OK;
}

}  // namespace

extern "C" int md_kinetic_energy_noalloc(int64_t n, const double* vel, const int32_t* species,
                                         const double* mass, int32_t n_species, double* ke_out, void* stream) {
    if (n < 0 || n > NOALLOC_MAX_ATOMS) return MD_ERR_ARG;
    if (!ke_out || !mass || n_species < 1 || n_species > mdgb::MAX_SPECIES) return MD_ERR_ARG;
    if (n > 0 && !vel) return MD_ERR_ARG;
    double* partials = nullptr;
    int rc = partials_for_current_device(&partials);
    if (rc) return rc;
    NoallocMass m{};
    for (int a = 0; a < n_species; ++a) m.m[a] = mass[a];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    long long nparts = (n + 2047) / 2048;
    if (nparts < 1) nparts = 1;
    if (nparts > NOALLOC_MAX_PARTS) nparts = NOALLOC_MAX_PARTS;
    const long long chunk = n > 0 ? (n + nparts - 1) / nparts : 1;
    // cudaLaunchKernel reports each launch's own status, so an error left pending by the
    // caller's earlier work is neither taken for this call's nor cleared by it
    int nsp = n_species, np_i = (int)nparts;
    long long n_arg = n;
    const double* vel_arg = vel;
    const int32_t* sp_arg = species;
    void* a1[] = {&n_arg, &vel_arg, &sp_arg, &nsp, &m, const_cast<long long*>(&chunk), &partials};
    if (cudaLaunchKernel((const void*)k_ke_partials, dim3((unsigned)nparts), dim3(NOALLOC_THREADS), a1, 0, st) !=
        cudaSuccess)
        return MD_ERR_CUDA;
    void* a2[] = {&partials, &np_i, &ke_out};
    if (cudaLaunchKernel((const void*)k_ke_final, dim3(1), dim3(NOALLOC_THREADS), a2, 0, st) != cudaSuccess)
        return MD_ERR_CUDA;
    return MD_OK;
}
