// Power reduction that allocates nothing.
//
// Some callers cannot call cudaMalloc: a host framework that owns a fixed
// device-memory budget and hands out only the buffers it has already set
// aside, or a latency-critical loop in which an allocation (which can wait on
// the whole device and can fail once the memory is committed) is not allowed.
// shg_field_powers_noalloc serves them: it computes the powers of fields the
// caller already holds, into an output the caller already holds, and keeps
// its per-block partial sums in the file-scope array below, which every GPU
// that loads this library holds until the process exits.
#include <mutex>

#include "plan.h"

namespace shg {

constexpr int kNaBlocks = 32;        // partial-sum blocks per instance
constexpr int kNaThreads = 256;
constexpr int kNaMaxInstances = 1024;
constexpr size_t kNaScratchDoubles = size_t(kNaMaxInstances) * kNaBlocks * 2;  // 512 KiB

// Shared by every call on a device: calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[kNaScratchDoubles];

static std::mutex g_na_mu;
static double* g_na_ptr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
static shg_status_t scratch_on_current_device(double** out) {
    int dev = 0;
    SHG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SHG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        SHG_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return SHG_OK;
}

// Pass 1: every block writes both of its partial sums (so nothing needs to be
// cleared between calls).  grid = (kNaBlocks, n_inst).
template <class C>
__global__ void k_na_partial(const C* __restrict__ fields, size_t npts, double* __restrict__ scr) {
    const C* f = fields + size_t(blockIdx.y) * 2 * npts;
    double aF = 0, aS = 0;
    for (size_t i = blockIdx.x * size_t(kNaThreads) + threadIdx.x; i < npts;
         i += size_t(gridDim.x) * kNaThreads) {
        const C u = f[i], v = f[npts + i];
        aF += double(u.x) * u.x + double(u.y) * u.y;
        aS += double(v.x) * v.x + double(v.y) * v.y;
    }
    __shared__ double sa[kNaThreads], sb[kNaThreads];
    sa[threadIdx.x] = aF;
    sb[threadIdx.x] = aS;
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = scr + (size_t(blockIdx.y) * kNaBlocks + blockIdx.x) * 2;
        o[0] = sa[0];
        o[1] = sb[0];
    }
}

// Pass 2: fixed-order sum of the partials of each instance.  grid = n_inst.
__global__ void k_na_final(const double* __restrict__ scr, double cF, double cS,
                           double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    const double* s = scr + size_t(blockIdx.x) * kNaBlocks * 2;
    double aF = 0, aS = 0;
    for (int b = 0; b < kNaBlocks; ++b) {
        aF += s[2 * b];
        aS += s[2 * b + 1];
    }
    out[2 * blockIdx.x] = cF * aF;
    out[2 * blockIdx.x + 1] = cS * aS;
}

}  // namespace shg

using namespace shg;

extern "C" shg_status_t shg_field_powers_noalloc(const void* fields_dev, int nx, int ny,
                                                 int n_inst, int fp64, double lx, double ly,
                                                 double n_f, double n_sh, double* powers_dev,
                                                 shg_stream_t stream) {
    if (!fields_dev || !powers_dev || nx <= 0 || ny <= 0 || !(lx > 0) || !(ly > 0))
        return SHG_ERR_INVALID_ARG;
    if (n_inst < 1 || n_inst > kNaMaxInstances) {
        cuda_fail(cudaErrorInvalidValue, "shg_field_powers_noalloc: n_inst must be in [1, 1024]");
        return SHG_ERR_INVALID_ARG;
    }
    double* scr = nullptr;
    shg_status_t r = scratch_on_current_device(&scr);
    if (r != SHG_OK) return r;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t npts = size_t(nx) * ny;
    const double dxdy = (lx / nx) * (ly / ny);
    const double cF = 0.5 * kEps0 * kCLight * n_f * dxdy, cS = 0.5 * kEps0 * kCLight * n_sh * dxdy;
    dim3 grid(kNaBlocks, n_inst);
    if (fp64)
        k_na_partial<double2><<<grid, kNaThreads, 0, st>>>(
            static_cast<const double2*>(fields_dev), npts, scr);
    else
        k_na_partial<float2><<<grid, kNaThreads, 0, st>>>(static_cast<const float2*>(fields_dev),
                                                          npts, scr);
    k_na_final<<<n_inst, 32, 0, st>>>(scr, cF, cS, powers_dev);
    SHG_CK(cudaGetLastError());
    return SHG_OK;
}
