// cslbm_total_mass_static: the total-mass reduction with its scratch in a
// file-scope device array instead of the context's workspace.
//
// Who needs it: code that may not allocate device memory at the point where
// it wants the mass -- a real-time loop or a host callback that must not
// enter the CUDA allocator, a plugin running under a framework that owns
// every allocation, or code that runs while a memory pool is being
// resized -- and that must not disturb the context's own reduction scratch
// (which cslbm_total_mass and cslbm_wall_force reuse).  This entry point
// calls no cudaMalloc, cudaFree or allocating library routine.
//
// The scratch is kMaxPartials FP64 partial sums (2 MiB) that every GPU
// loading the library holds until the process exits.  Each 256-node block
// of the lattice writes one partial; a single block then adds them up in a
// fixed order, so the result is the same bit for bit on every call (the
// workspace version adds with atomics).  Every partial a call reads is
// written by that call, so nothing needs clearing; the array keeps the last
// call's contents, and calls that overlap on the GPU (on several streams or
// several contexts of one device) race on it.
#include <cstdio>
#include <mutex>
#include <string>

#include "ctx.h"
#include "lbm_device.cuh"
#include "make_lat.h"

namespace {

constexpr int kBlock = 256;
constexpr long long kMaxPartials = 1LL << 18;  // at most 67,108,864 nodes per call
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_mass_scratch[kMaxPartials + 1];  // partials, then the total

double* g_scratch_ptr[kMaxDevices];
std::once_flag g_scratch_once[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

template <class S, class R>
__global__ void __launch_bounds__(kBlock) k_mass_partials(cslbm::Lat L, const S* __restrict__ P,
                                                          const R* __restrict__ hist, const R* __restrict__ geo,
                                                          double* partials)
{
    using namespace cslbm;
    const long long v = blockIdx.x * (long long)kBlock + threadIdx.x;
    double val = 0.0;
    if (v < L.N) {
        const int x = (int)(v % L.n[0]);
        const long long r = v / L.n[0];
        const int y = (int)(r % L.n[1]), z = (int)(r / L.n[1]);
        R s[Q];
        node_pops<S, R>(L, P, hist, geo, x, y, z, s);
        R m0 = R(0);
#pragma unroll
        for (int l = 0; l < Q; l++) m0 += s[l];
        const R sg = geo[v];
        const R rho = sg * (R(1) + m0) + R(0.5) * hist[v];  // rho = sqrt(g) sum h + A'/2
        val = double(sg) * double(rho);
    }
    __shared__ double part[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBlock / 32; w++) t += part[w];
        partials[blockIdx.x] = t;
    }
}

// fixed-order sum of n partials into partials[kMaxPartials]
__global__ void __launch_bounds__(kBlock) k_sum_partials(double* partials, long long n)
{
    __shared__ double part[kBlock];
    double t = 0.0;
    for (long long i = threadIdx.x; i < n; i += kBlock) t += partials[i];
    part[threadIdx.x] = t;
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[kMaxPartials] = part[0];
}

template <class S, class R>
void launch(const cslbm_ctx* c, double* partials, unsigned nb)
{
    k_mass_partials<S, R><<<nb, kBlock, 0, c->stream>>>(cslbm::make_lat(c), (const S*)c->P[c->pc], (const R*)c->H[c->hc],
                                                       (const R*)c->G[c->gc], partials);
}

}  // namespace

extern "C" {

cslbm_status cslbm_total_mass_static(cslbm_ctx* c, double* out)
{
    if (!c || !out) return cslbm_record_error(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return cslbm_record_error(CSLBM_ESTATE, "no state");
    const long long nb = (c->N + kBlock - 1) / kBlock;
    if (nb > kMaxPartials) {
        char m[160];
        snprintf(m, sizeof m, "lattice of %lld nodes exceeds the static scratch of cslbm_total_mass_static "
                              "(at most %lld nodes)", c->N, kMaxPartials * kBlock);
        return cslbm_record_error(CSLBM_EINVAL, m);
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || dev != c->device)
        return cslbm_record_error(CSLBM_EINVAL, "the context's device must be the current device");
    // once per device, with that device current: the device address of the array
    std::call_once(g_scratch_once[dev], [dev] {
        g_scratch_err[dev] = cudaGetSymbolAddress((void**)&g_scratch_ptr[dev], g_mass_scratch);
    });
    if (g_scratch_err[dev] != cudaSuccess)
        return cslbm_record_error(CSLBM_ECUDA, (std::string("cudaGetSymbolAddress failed: ") +
                                                cudaGetErrorString(g_scratch_err[dev])).c_str());
    double* partials = g_scratch_ptr[dev];
    switch (c->p.storage) {
    case CSLBM_FP32: launch<float, float>(c, partials, (unsigned)nb); break;
    case CSLBM_FP16S: launch<__half, float>(c, partials, (unsigned)nb); break;
    case CSLBM_BF16S: launch<__nv_bfloat16, float>(c, partials, (unsigned)nb); break;
    default: launch<double, double>(c, partials, (unsigned)nb); break;
    }
    k_sum_partials<<<1, kBlock, 0, c->stream>>>(partials, nb);
    c->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, partials + kMaxPartials, sizeof(double), cudaMemcpyDeviceToHost,
                                              c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cslbm_record_error(CSLBM_ECUDA, (std::string("cslbm_total_mass_static: ") + cudaGetErrorString(e)).c_str());
    return CSLBM_OK;
}

}  // extern "C"
