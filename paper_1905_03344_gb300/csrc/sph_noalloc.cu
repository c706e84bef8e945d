// sph_noalloc.cu -- sph_conserved_noalloc: the conserved sums of particle
// arrays the caller already holds on the device, computed without allocating
// anything.  For callers that cannot call cudaMalloc: code running while a
// stream is being captured into a CUDA graph, an allocator-owning host
// framework that forbids other allocations, or a process that has handed
// all device memory to its own pool.
//
// The per-block partial sums live in a file-scope device array of fixed size
// (kStaticBlocks x 8 doubles, 256 KB), which every GPU that loads the
// library keeps until the process exits.  Host code cannot use the array's
// name as a device address; its address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device, and passed to the kernels.  That first call should therefore
// come before any stream capture.  The address is kept for the life of the
// process: a device reset (cudaDeviceReset, or a new primary context on that
// device) makes it stale, and the entry point must not be called on that
// device afterwards.  All calls share the one array: it is
// overwritten by every call (each block writes its own slot before the final
// sum reads it, so nothing needs clearing), and calls whose kernels overlap on
// the GPU race on it.
#include <mutex>
#include <string>

#include "sph_internal.cuh"

namespace {

constexpr int kStaticBlocks = 4096;                   // partial-sum slots
constexpr int kStaticChunk = 4096;                    // particles per block
constexpr int64_t kStaticMaxN = (int64_t)kStaticBlocks * kStaticChunk;  // 16,777,216
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_partials[kStaticBlocks * 8];

std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};
thread_local std::string g_noalloc_error;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one block per chunk of kStaticChunk particles: the 7 sums of the chunk into
// the block's slot (M, Px, Py, Pz, Lz, Ekin, Eint)
__global__ void __launch_bounds__(256) k_cons_partials(int64_t n, const double* x, const double* y,
                                                       const double* vx, const double* vy, const double* vz,
                                                       const double* m, const double* u, double* part)
{
    __shared__ double sh[7][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * kStaticChunk;
    const int64_t b1 = b0 + kStaticChunk < n ? b0 + kStaticChunk : n;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double mi = m[i], vxi = vx[i], vyi = vy[i], vzi = vz[i];
        acc[0] += mi;
        acc[1] += mi * vxi;
        acc[2] += mi * vyi;
        acc[3] += mi * vzi;
        acc[4] += mi * (x[i] * vyi - y[i] * vxi);
        acc[5] += 0.5 * mi * (vxi * vxi + vyi * vyi + vzi * vzi);
        acc[6] += mi * u[i];
    }
    for (int q = 0; q < 7; q++) acc[q] = warp_sum(acc[q]);
    if (lane == 0)
        for (int q = 0; q < 7; q++) sh[q][warp] = acc[q];
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[threadIdx.x][w];
        part[(int64_t)blockIdx.x * 8 + threadIdx.x] = s;
    }
}

// seven threads: compensated sum of the block slots in block order
__global__ void k_cons_final(int nblocks, const double* part, double* out)
{
    const int q = threadIdx.x;
    if (q >= 7) return;
    double s = 0.0, c = 0.0;
    for (int b = 0; b < nblocks; b++) {
        const double v = part[(int64_t)b * 8 + q];
        const double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    out[q] = s + c;
}

sph_status noalloc_fail(sph_status s, const std::string& msg)
{
    g_noalloc_error = msg;
    return s;
}

}  // namespace

extern "C" sph_status sph_conserved_noalloc(int64_t n, const double* x, const double* y, const double* vx,
                                            const double* vy, const double* vz, const double* m,
                                            const double* u, double* out, void* cuda_stream)
{
    if (n < 0 || n > kStaticMaxN)
        return noalloc_fail(SPH_EINVAL, "sph_conserved_noalloc: n must be in [0, 16777216] (fixed scratch)");
    if (!out) return noalloc_fail(SPH_EINVAL, "sph_conserved_noalloc: out is NULL");
    if (n > 0 && (!x || !y || !vx || !vy || !vz || !m || !u))
        return noalloc_fail(SPH_EINVAL, "sph_conserved_noalloc: NULL field pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SPH_ECUDA, std::string("sph_conserved_noalloc: no usable device: ") +
                                           cudaGetErrorString(e));
    double* part = nullptr;
    {
        // once per device, with that device current: the device address of the
        // file-scope scratch array
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || !p)
                return noalloc_fail(SPH_ECUDA, std::string("sph_conserved_noalloc: cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
            g_partials_addr[dev] = (double*)p;
        }
        part = g_partials_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nblocks = (int)((n + kStaticChunk - 1) / kStaticChunk);
    if (nblocks > 0) k_cons_partials<<<nblocks, 256, 0, st>>>(n, x, y, vx, vy, vz, m, u, part);
    k_cons_final<<<1, 32, 0, st>>>(nblocks, part, out);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(SPH_ECUDA, std::string("sph_conserved_noalloc: launch: ") + cudaGetErrorString(e));
    return SPH_OK;
}

extern "C" const char* sph_noalloc_last_error(void) { return g_noalloc_error.c_str(); }
