// Allocation-free variant of the deflation projection y = P x = x - S Z K Z^T x.
//
// Why it exists: some callers of this library cannot allocate device memory
// at the point where they need the projection -- real-time loops (a time
// stepper calling the projection every step) that must not hit the
// allocator's latency or the device-wide synchronisation cudaMalloc and
// cudaFree can cause, and host applications that hand the library a fixed
// device-memory budget up front and own every allocation themselves.  smpm_apply() may grow the handle's workspace on first use;
// smpm_apply_deflation_noalloc() never allocates: its only scratch (the coarse
// vectors q = Z^T x and c = K q) lives in the file-scope device array below,
// which every GPU that loads the library holds until the process exits.
//
// Limits and sharing: the scratch holds SMPM_NOALLOC_MAX_DOUBLES doubles and
// a call needs 2 * nrhs * d of them (d = coarse dimension); larger requests
// are rejected.  All calls on a device share the one array and it keeps the
// last call's contents; every entry a call reads is written by that call
// first, so nothing needs clearing, but calls whose kernels overlap on the
// GPU (different streams, or different handles on one stream without
// ordering) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/smpm.h"
#include "kernels.h"
#include "smpm_internal.h"

namespace smpm {

static constexpr long long kNoallocMax = SMPM_NOALLOC_MAX_DOUBLES;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocMax];

static constexpr int kNB = 256;

__device__ __forceinline__ double nwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// q[r][t ng + g] = sum of x over group g of both faces of interface t
// (x in the unpadded interface order: interface t is [2 t fz, (2 t + 2) fz)).
__global__ void na_restrict_kernel(DeflView v, int R, const double* __restrict__ x, double* __restrict__ q) {
    const int r = blockIdx.y;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wg >= v.d || r >= R) return;
    const int t = wg / v.ng, gi = wg % v.ng, gs = v.fz / v.ng;
    const long long off = (long long)r * v.k + (long long)(2 * t) * v.fz + (long long)gi * gs;
    double s = 0.0;
    for (int z = lane; z < gs; z += 32) s += x[off + z] + x[off + v.fz + z];
    s = nwarp_sum(s);
    if (lane == 0) q[(long long)r * v.d + wg] = s;
}

// c[r][i] = sum_j K[i][j] q[r][j]
__global__ void na_coarse_kernel(DeflView v, int R, const double* __restrict__ q, double* __restrict__ c) {
    const int r = blockIdx.y;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= v.d || r >= R) return;
    const double* Ki = v.K + (long long)i * v.d;
    const double* qr = q + (long long)r * v.d;
    double s = 0.0;
    for (int j = lane; j < v.d; j += 32) s = fma(Ki[j], qr[j], s);
    s = nwarp_sum(s);
    if (lane == 0) c[(long long)r * v.d + i] = s;
}

// y = x - S Z c.  Unpadded position i is face F = i / fz + 1 of the strip-face
// numbering (face 2 s + side); Z c is c_{t,g} on both faces of interface t and S
// adds the G row sums rho of the two strips touching it.
// x and y may be the same buffer (each thread reads and then writes its own
// element), so neither is marked __restrict__.
__global__ void na_correct_kernel(DeflView v, int R, const double* x, const double* __restrict__ c, double* y) {
    const int r = blockIdx.y;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.k || r >= R) return;
    const int fz = v.fz, ng = v.ng, gs = fz / ng;
    const long long fz2 = 2LL * fz;
    const int F = (int)(i / fz) + 1, Z = (int)(i % fz);
    const int strip = F >> 1, side = F & 1;
    const double* cr = c + (long long)r * v.d;
    double val;
    if (side == 1) {          // east face of `strip`, interface t = strip
        const int t = strip, cl = v.strip_cls[strip + 1];
        const double* rL = v.rho + (long long)(cl * 2 + 0) * ng * fz2;
        const double* rR = v.rho + (long long)(cl * 2 + 1) * ng * fz2;
        val = cr[t * ng + Z / gs];
        for (int g = 0; g < ng; ++g) {
            val = fma(cr[t * ng + g], rL[g * fz2 + Z], val);
            if (t + 1 <= v.mx - 2) val = fma(cr[(t + 1) * ng + g], rR[g * fz2 + Z], val);
        }
    } else {                  // west face of `strip`, interface t = strip - 1
        const int t = strip - 1, cl = v.strip_cls[strip - 1];
        const double* rL = v.rho + (long long)(cl * 2 + 0) * ng * fz2 + fz;
        const double* rR = v.rho + (long long)(cl * 2 + 1) * ng * fz2 + fz;
        val = cr[t * ng + Z / gs];
        for (int g = 0; g < ng; ++g) {
            if (t >= 1) val = fma(cr[(t - 1) * ng + g], rL[g * fz2 + Z], val);
            val = fma(cr[t * ng + g], rR[g * fz2 + Z], val);
        }
    }
    y[(long long)r * v.k + i] = x[(long long)r * v.k + i] - val;
}

// Device address of the scratch array, looked up once per device (the
// cache assumes the device's primary context lives as long as the process:
// after cudaDeviceReset the module is loaded again and the address must be
// looked up again, which this cache would not do).
static std::mutex g_na_mutex;
static double* g_na_ptr[64] = {nullptr};

static int noalloc_scratch(double** out, std::string& msg) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return SMPM_ECUDA; }
    if (dev < 0 || dev >= 64) { msg = "device index above 63"; return SMPM_EINVAL; }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return SMPM_ECUDA;
        }
        g_na_ptr[dev] = (double*)p;
    }
    *out = g_na_ptr[dev];
    return SMPM_OK;
}

static bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace smpm

extern "C" int smpm_apply_deflation_noalloc(smpm_handle h, int nrhs, const double* x, double* y) {
    using namespace smpm;
    std::string msg;
    DeflView v;
    if (!h || !x || !y || nrhs <= 0) {
        set_last_error("smpm_apply_deflation_noalloc: null handle or buffer, or nrhs <= 0");
        return SMPM_EINVAL;
    }
    if (!deflation_view(h, &v, msg)) {
        set_last_error(msg);
        return SMPM_EINVAL;
    }
    const long long need = 2LL * nrhs * v.d;
    if (need > kNoallocMax) {
        set_last_error("smpm_apply_deflation_noalloc: 2 * nrhs * d = " + std::to_string(need) +
                       " doubles of coarse scratch exceed the fixed " + std::to_string(kNoallocMax) +
                       " (SMPM_NOALLOC_MAX_DOUBLES); use fewer right-hand sides per call");
        return SMPM_EINVAL;
    }
    if (!on_device(x) || !on_device(y)) {
        set_last_error("smpm_apply_deflation_noalloc: x and y must be device pointers");
        return SMPM_EINVAL;
    }
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch, msg);
    if (rc != SMPM_OK) {
        set_last_error(msg);
        return rc;
    }
    double* q = scratch;
    double* c = scratch + (long long)nrhs * v.d;
    dim3 gw((unsigned)((v.d * 32 + kNB - 1) / kNB), nrhs);
    na_restrict_kernel<<<gw, kNB, 0, v.stream>>>(v, nrhs, x, q);
    na_coarse_kernel<<<gw, kNB, 0, v.stream>>>(v, nrhs, q, c);
    dim3 gk((unsigned)((v.k + kNB - 1) / kNB), nrhs);
    na_correct_kernel<<<gk, kNB, 0, v.stream>>>(v, nrhs, x, c, y);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("smpm_apply_deflation_noalloc launch: ") + cudaGetErrorString(e));
        return SMPM_ECUDA;
    }
    set_last_error("");
    return SMPM_OK;
}
