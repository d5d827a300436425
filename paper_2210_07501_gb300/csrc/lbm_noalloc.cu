// lbm_noalloc.cu -- the field reduction (mass, velocity-change and velocity norms,
// non-finite count) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that enqueues work while a stream is being
// captured into a CUDA graph, or a plugin / custom call inside a framework that owns every
// device allocation and only hands it buffers.  lbm_reduce_fields_noalloc serves them: the
// caller passes the input fields and the output array, and the per-block partial sums live
// in the fixed array below, which every GPU that loads this library keeps until the
// process exits.  No cudaMalloc, cudaFree or allocating library routine is called.
#include <mutex>

#include "../../include/lbm_gb300.h"
#include "lbm_internal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_BLOCKS = 304;  // 2 x 152 SMs; the partials need NA_BLOCKS * 4 doubles

// Scratch for the block partials: 304 x 4 doubles = 9.5 KiB per device.
static __device__ __align__(256) double g_noalloc_partials[NA_BLOCKS * 4];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double *g_partials_ptr[MAX_DEVICES] = {nullptr};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Same launch shape, per-thread assignment and summation order as the handle's reduction,
// so both give identical sums for identical fields.
__global__ void __launch_bounds__(NA_THREADS)
noalloc_partial_kernel(const double *__restrict__ phi, const double *__restrict__ u, const double *__restrict__ v,
                       const double *__restrict__ T, const double *__restrict__ up, const double *__restrict__ vp,
                       long long N, double *__restrict__ partials)
{
    double m = 0.0, du2 = 0.0, u2 = 0.0, bad = 0.0;
    for (long long i = blockIdx.x * (long long)NA_THREADS + threadIdx.x; i < N; i += (long long)gridDim.x * NA_THREADS) {
        const double p = phi[i], a = u[i], b = v[i], t = T[i];
        const double pa = up ? up[i] : 0.0, pb = vp ? vp[i] : 0.0;
        m += p;
        du2 += (a - pa) * (a - pa) + (b - pb) * (b - pb);
        u2 += a * a + b * b;
        if (!isfinite(p) || !isfinite(a) || !isfinite(b) || !isfinite(t)) bad += 1.0;
    }
    __shared__ double sh[4][NA_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    m = warp_sum(m);
    du2 = warp_sum(du2);
    u2 = warp_sum(u2);
    bad = warp_sum(bad);
    if (lane == 0) {
        sh[0][wid] = m;
        sh[1][wid] = du2;
        sh[2][wid] = u2;
        sh[3][wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) s += sh[threadIdx.x][w];
        partials[blockIdx.x * 4 + threadIdx.x] = s;   // every slot is written: no zeroing needed
    }
}

__global__ void noalloc_final_kernel(const double *__restrict__ partials, int nblk, double *__restrict__ result)
{
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partials[b * 4 + threadIdx.x];
        result[threadIdx.x] = s;
    }
}

// Once per device, with that device current: the device address of the scratch array.
int partials_for_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return LBM_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) return LBM_ECUDA;
        g_partials_ptr[dev] = (double *)p;
    }
    *out = g_partials_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_fields_noalloc(const double *phi, const double *u, const double *v, const double *T,
                                         const double *u_prev, const double *v_prev, int64_t n_nodes,
                                         double *result, void *stream)
{
    if (!phi || !u || !v || !T || !result) return LBM_EINVAL;
    if (n_nodes < 1 || n_nodes > LBM_NOALLOC_MAX_NODES) return LBM_EINVAL;
    if ((u_prev == nullptr) != (v_prev == nullptr)) return LBM_EINVAL;
    double *partials = nullptr;
    int rc = partials_for_current_device(&partials);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    noalloc_partial_kernel<<<NA_BLOCKS, NA_THREADS, 0, s>>>(phi, u, v, T, u_prev, v_prev, (long long)n_nodes, partials);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    noalloc_final_kernel<<<1, 32, 0, s>>>(partials, NA_BLOCKS, result);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}
