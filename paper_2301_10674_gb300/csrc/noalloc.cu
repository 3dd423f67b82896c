// Allocation-free FP64 reduction of caller-owned lattice fields.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or
// arena that another framework owns, or code that may only touch memory it was
// handed. This entry point computes the liquid mass and momentum of fields the
// caller already holds on the device (for example fields exported with
// fslbm_get_fields) and needs no fslbm handle: its scratch is a fixed array in
// the library's device image, not an allocation.
#include <cstdint>

#include "fslbm.h"
#include "fslbm_dev.cuh"

namespace {

constexpr int NA_CHUNK = 65536;    // cells per block of the reduction
constexpr int NA_PARTIALS = 4096;  // blocks of partial sums the scratch holds
constexpr int NA_THREADS = 256;

// Scratch: one row of 4 partial sums per block. It lives as long as the
// library is loaded on each device that uses it, and every call shares it.
static __device__ __align__(256) double na_scratch[NA_PARTIALS * 4];

// Each block reduces its own chunk of cells in a fixed order and stores one
// row of partials; the final pass adds the rows in block order, so the result
// does not depend on scheduling.
__global__ void k_na_partials(const double* __restrict__ pdf, const uint8_t* __restrict__ type,
                              const double* __restrict__ mass, long long n, double gx, double gy, double gz,
                              double* scratch) {
    __shared__ double sh[4][NA_THREADS];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long lo = (long long)blockIdx.x * NA_CHUNK;
    const long long hi = lo + NA_CHUNK < n ? lo + NA_CHUNK : n;
    for (long long c = lo + threadIdx.x; c < hi; c += NA_THREADS) {
        const int t = type[c] & 3;
        if (t != FSLBM_LIQUID && t != FSLBM_INTERFACE) continue;
        double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
        for (int q = 0; q < 27; ++q) {
            const double v = pdf[(long long)q * n + c];
            rho += v;
            jx += fsl::cx(q) * v;
            jy += fsl::cy(q) * v;
            jz += fsl::cz(q) * v;
        }
        acc[0] += t == FSLBM_LIQUID ? rho : mass[c];
        acc[1] += jx - 0.5 * rho * gx;
        acc[2] += jy - 0.5 * rho * gy;
        acc[3] += jz - 0.5 * rho * gz;
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int off = NA_THREADS / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x < 4) scratch[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_na_final(const double* __restrict__ scratch, int blocks, double* out) {
    if (threadIdx.x >= 4) return;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += scratch[4 * b + threadIdx.x];
    out[threadIdx.x] = s;
}

}  // namespace

extern "C" int fslbm_reduce_fields_noalloc(const double* pdf, const uint8_t* type, const double* mass,
                                           int64_t ncells, const double g[3], double* out, void* cuda_stream) {
    if (!pdf || !type || !mass || !g || !out || ncells <= 0) return FSLBM_EINVAL;
    if (ncells > (int64_t)NA_CHUNK * NA_PARTIALS) return FSLBM_ECAPACITY;
    // Device address of the scratch array on the current device. In host code
    // na_scratch names a host-side stand-in, not device memory, so the address
    // is looked up (a host-side table query once the device image is loaded;
    // the first call on a device loads it). Looking it up on every call keeps
    // no host state between calls, so a device reset in between does no harm
    // and concurrent host threads share nothing.
    double* scratch = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&scratch), na_scratch) != cudaSuccess || !scratch) {
        cudaGetLastError();
        return FSLBM_EDEVICE;
    }
    // a launch error pending from earlier, unrelated work is not this call's
    cudaGetLastError();
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = (int)((ncells + NA_CHUNK - 1) / NA_CHUNK);
    // every block writes its own row, so nothing has to be cleared first
    k_na_partials<<<blocks, NA_THREADS, 0, st>>>(pdf, type, mass, (long long)ncells, g[0], g[1], g[2], scratch);
    if (cudaGetLastError() != cudaSuccess) return FSLBM_EDEVICE;
    k_na_final<<<1, 32, 0, st>>>(scratch, blocks, out);
    if (cudaGetLastError() != cudaSuccess) return FSLBM_EDEVICE;
    return FSLBM_OK;
}
