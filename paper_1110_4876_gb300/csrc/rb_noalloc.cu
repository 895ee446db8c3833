// rb_noalloc.cu -- energy and momentum sums for callers that cannot allocate
// device memory.
//
// rb_energy_sums_noalloc is the allocation-free counterpart of the per-block
// reduction behind rb_energy: the caller passes the particle arrays and a
// 7-double output, both in device memory, and the per-block partial sums
// live in a fixed array in the library's own device memory.  Callers that
// cannot call cudaMalloc (a host process whose device memory is owned by
// another runtime's pool or budget, a latency-bound loop that must not hit
// the implicit synchronisation of an allocation) can still use it.
#include <mutex>
#include <string>

#include "rb.h"
#include "rb_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int kTile = kThreads * kPerThread;            // particles per block
constexpr int kMaxBlocks = 8192;                        // partial-sum slots
constexpr int64_t kMaxParticles = (int64_t)kMaxBlocks * kTile;  // 16,777,216
constexpr int kMaxDevices = 64;

// Per-block partial sums: 7 x 8192 doubles = 448 KiB on every GPU that loads
// the library, held until the process exits.  Every call overwrites the
// slots it reads, so nothing has to start at zero; calls that overlap on the
// GPU share this array and race.
static __device__ __align__(256) double g_energy_scratch[7 * kMaxBlocks];

double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array on device `dev`, which must be the
// current device (looked up once per device; the host-side symbol itself is
// not a device address).  The cached address belongs to the context that
// was current at the lookup: a caller that resets the device
// (cudaDeviceReset) and keeps using the library in a new context gets a
// stale address, which this library does not detect.
cudaError_t scratch_for_device(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Terms of Sect. 6.2 (and the Hill tidal/vertical terms for SEI), one partial
// per block: K, U_tidal, W = m phi / 2, Px, Py, Pz, count.
__global__ void __launch_bounds__(kThreads) k_energy_noalloc(
    int n, const double* __restrict__ m, const double* __restrict__ x,
    const double* __restrict__ z, const double* __restrict__ vx, const double* __restrict__ vy,
    const double* __restrict__ vz, const double* __restrict__ phi, int sei, double omega2,
    double omega_z2, double* __restrict__ partials) {
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    const int base = blockIdx.x * kTile + threadIdx.x;
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {
        const int i = base + r * kThreads;
        if (i >= n) break;
        const double mi = m[i], u = vx[i], v = vy[i], w = vz[i];
        s[0] += 0.5 * mi * (u * u + v * v + w * w);
        if (sei) s[1] += mi * (0.5 * omega_z2 * (z[i] * z[i]) - 1.5 * omega2 * (x[i] * x[i]));
        if (phi) s[2] += 0.5 * mi * phi[i];
        s[3] += mi * u;
        s[4] += mi * v;
        s[5] += mi * w;
        s[6] += 1.0;
    }
    __shared__ double red[7][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 7; q++) {
        double t = s[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double t = 0.0;
        for (int k = 0; k < kThreads / 32; k++) t += red[threadIdx.x][k];
        partials[threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// Sum of the partials in block order (the same result for the same inputs).
__global__ void k_energy_noalloc_final(const double* __restrict__ partials, int nblocks,
                                       double* __restrict__ out) {
    const int q = threadIdx.x;
    if (q >= 7) return;
    double t = 0.0;
    for (int k = 0; k < nblocks; k++) t += partials[q * nblocks + k];
    out[q] = t;
}

}  // namespace

extern "C" int rb_energy_sums_noalloc(int64_t n, const double* m, const double* x, const double* z,
                                      const double* vx, const double* vy, const double* vz,
                                      const double* phi, int integrator, double omega,
                                      double omega_z, double* out, void* cuda_stream) {
    if (n < 0 || n > kMaxParticles) {
        rb::set_global_error("rb_energy_sums_noalloc: n must be in [0, 16777216] (the size of its "
                             "fixed partial-sum array)");
        return RB_ERR_ARG;
    }
    if (!out || (n > 0 && (!m || !vx || !vy || !vz)) ||
        (integrator == RB_INT_SEI && n > 0 && (!x || !z))) {
        rb::set_global_error("rb_energy_sums_noalloc: null array");
        return RB_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        rb::set_global_error(std::string("rb_energy_sums_noalloc: cudaGetDevice: ") +
                             cudaGetErrorString(e));
        return RB_ERR_CUDA;
    }
    if (s) {
        int sdev = -1;
        e = cudaStreamGetDevice(s, &sdev);
        if (e != cudaSuccess) {
            rb::set_global_error(std::string("rb_energy_sums_noalloc: cudaStreamGetDevice: ") +
                                 cudaGetErrorString(e));
            return RB_ERR_CUDA;
        }
        if (sdev != dev) {
            rb::set_global_error("rb_energy_sums_noalloc: cuda_stream belongs to another device "
                                 "than the current one");
            return RB_ERR_ARG;
        }
    }
    double* scratch = nullptr;
    e = scratch_for_device(dev, &scratch);
    if (e != cudaSuccess) {
        rb::set_global_error(std::string("rb_energy_sums_noalloc: cudaGetSymbolAddress: ") +
                             cudaGetErrorString(e));
        return RB_ERR_CUDA;
    }
    const int nblocks = n > 0 ? (int)((n + kTile - 1) / kTile) : 1;
    const double oz = omega_z > 0.0 ? omega_z : omega;
    // A launch error left over from earlier work on this thread (by this
    // library or another) is cleared first, so that the check below reports
    // only these two launches.
    (void)cudaGetLastError();
    k_energy_noalloc<<<nblocks, kThreads, 0, s>>>((int)n, m, x, z, vx, vy, vz, phi,
                                                  integrator == RB_INT_SEI, omega * omega, oz * oz,
                                                  scratch);
    k_energy_noalloc_final<<<1, 32, 0, s>>>(scratch, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        rb::set_global_error(std::string("rb_energy_sums_noalloc: kernel launch: ") +
                             cudaGetErrorString(e));
        return RB_ERR_CUDA;
    }
    return RB_OK;
}
