// lbm_aux.cu -- initialisation, reductions and state conversion kernels of the GB300
// coupled LB library (arXiv 2210.07501).
#include <math.h>

#include "lbm_internal.h"

namespace lbm {

// ---- initialisation: default fields (Sec. 3 tanh profile; rest; T_ref; uniform p) ----
__global__ void init_defaults_kernel(double *macro, int nx, int ny, double b, double W, double T_ref, int defaults)
{
    const long long N = (long long)nx * ny;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const int j = int(m / nx);
        const double y = j + 0.5;
        if (defaults & 1) macro[m] = 0.5 + 0.5 * tanh(2.0 * (y - b) / W);
        if (defaults & 2) macro[N + m] = 0.0;
        if (defaults & 4) macro[2 * N + m] = 0.0;
        if (defaults & 8) macro[3 * N + m] = T_ref;
        if (defaults & 16) macro[4 * N + m] = 0.0;
    }
}

// Populations at the central-moment equilibrium of the given fields: phase field with the
// sharpening flux M theta n in its first moments (formed in FP64 and stored as its
// deviation from the reference populations r_a(y)), flow and energy lattices at their
// equilibria (no source), stored pressure = dp.
template <typename Real, typename Store, int QF, int QT>
__global__ void init_pop_kernel(const StepArgs<Real, Store> A)
{
    const int nx = A.nx, ny = A.ny;
    const long long N = (long long)nx * ny;
    const Phys<Real> &P = A.P;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const int y = int(m / nx), x = int(m - (long long)y * nx);
        const double *phiF = A.macro;
        auto phi_at = [&](int xx, int yy) -> double {
            return phiF[(long long)mirror_row_(yy, ny) * nx + wrap_(xx, nx)];
        };
        double s[3][3];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) s[dy + 1][dx + 1] = phi_at(x + dx, y + dy);
        double gx, gy, nxv, nyv;
        iso_grad_<double, 3>(s, 1, 1, gx, gy);
        unit_normal_(gx, gy, double(P.g2min), nxv, nyv);
        const double phi_d = s[1][1];
        const Real phi = Real(phi_d);
        const Real ux = Real(A.macro[N + m]), uy = Real(A.macro[2 * N + m]);
        const Real dT = Real(A.macro[3 * N + m] - double(P.T_ref));
        const Real dp = Real(A.macro[4 * N + m]);
        const Real c2 = Real(1.0 / 3.0);
        const long long o = (long long)y * A.pitch + x;
        // phase field, in FP64, minus the reference
        {
            double f[QF];
            const double uxd = A.macro[N + m], uyd = A.macro[2 * N + m];
            const double theta = double(P.W4) * phi_d * (1.0 - phi_d);
            const double mx = double(P.Mphi) * theta * nxv, my = double(P.Mphi) * theta * nyv, c2p = phi_d / 3.0;
            if constexpr (QF == 9) {
                const double k[9] = {phi_d, mx, my, c2p, c2p, 0.0, 0.0, 0.0, phi_d / 9.0};
                central_to_pop9_(k, k, uxd, uyd, f);
            } else {
                const double k[5] = {phi_d, mx, my, c2p, c2p};
                central_to_pop5_(k, k, uxd, uyd, f);
            }
#pragma unroll
            for (int a = 0; a < QF; ++a) {
                Real v = Real(f[a] - A.fref[a * ny + y]);
                if constexpr (scaled_<Store>()) v *= A.sf;
                st_(A.f_out + a * A.plane + o, v);
            }
        }
        // flow: deviation equilibrium dp Wc(u) + rho c^2 D(u)
        {
            const Real rho = P.rhoA + phi * P.drho;
            const Real ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
            const Real ax = c2 + ux2, ay = c2 + uy2, rc2 = rho * c2, d = rc2 - dp;
            const Real k[9] = {dp, ux * d, uy * d, dp * ax - rc2 * ux2, dp * ay - rc2 * uy2, -uxy * d, ax * uy * d,
                               ay * ux * d, dp * ax * ay - rc2 * (c2 * (ux2 + uy2) + ux2 * uy2)};
            Real g[9];
            central_to_pop9_(k, k, ux, uy, g);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                Real v = g[a];
                if constexpr (scaled_<Store>()) v *= A.sg;
                st_(A.g_out + a * A.plane + o, v);
            }
        }
        // energy: dT E + T_ref D(u)
        {
            Real h[QT];
            const Real Tr = P.T_ref, ux2 = ux * ux, uy2 = uy * uy;
            if constexpr (QT == 9) {
                const Real k[9] = {dT, Tr * ux, Tr * uy, c2 * dT - Tr * ux2, c2 * dT - Tr * uy2, -Tr * ux * uy,
                                   Tr * (c2 + ux2) * uy, Tr * (c2 + uy2) * ux,
                                   Real(1.0 / 9.0) * dT - Tr * (c2 * (ux2 + uy2) + ux2 * uy2)};
                central_to_pop9_(k, k, ux, uy, h);
            } else {
                const Real k[5] = {dT, Tr * ux, Tr * uy, c2 * dT - Tr * ux2, c2 * dT - Tr * uy2};
                central_to_pop5_(k, k, ux, uy, h);
            }
#pragma unroll
            for (int a = 0; a < QT; ++a) {
                Real v = h[a];
                if constexpr (scaled_<Store>()) v *= A.sh;
                st_(A.h_out + a * A.plane + o, v);
            }
        }
        A.dp_out[o] = dp;
    }
}

template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_init(const StepArgs<Real, Store> &A, double b, double W, int defaults, cudaStream_t s)
{
    const long long N = (long long)A.nx * A.ny;
    const int threads = 256;
    const int blocks = int((N + threads - 1) / threads < 4096 ? (N + threads - 1) / threads : 4096);
    if (defaults) {
        init_defaults_kernel<<<blocks, threads, 0, s>>>(A.macro, A.nx, A.ny, b, W, double(A.P.T_ref), defaults);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    init_pop_kernel<Real, Store, QF, QT><<<blocks, threads, 0, s>>>(A);
    return cudaGetLastError();
}

// ---- reductions: fixed launch shape and fixed-order final pass (deterministic) ----
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
int reduce_blocks() { return RED_BLOCKS; }

__device__ __forceinline__ double warp_sum_(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(RED_THREADS)
reduce_partial_kernel(const double *__restrict__ macro, double *__restrict__ uprev, long long N, int update,
                      double *__restrict__ partials)
{
    double m = 0.0, du2 = 0.0, u2 = 0.0, bad = 0.0;
    for (long long i = blockIdx.x * (long long)RED_THREADS + threadIdx.x; i < N; i += (long long)gridDim.x * RED_THREADS) {
        const double phi = macro[i], u = macro[N + i], v = macro[2 * N + i], T = macro[3 * N + i];
        const double up = uprev[i], vp = uprev[N + i];
        m += phi;
        du2 += (u - up) * (u - up) + (v - vp) * (v - vp);
        u2 += u * u + v * v;
        if (!isfinite(phi) || !isfinite(u) || !isfinite(v) || !isfinite(T)) bad += 1.0;
        if (update) {
            uprev[i] = u;
            uprev[N + i] = v;
        }
    }
    __shared__ double sh[4][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    m = warp_sum_(m);
    du2 = warp_sum_(du2);
    u2 = warp_sum_(u2);
    bad = warp_sum_(bad);
    if (lane == 0) {
        sh[0][wid] = m;
        sh[1][wid] = du2;
        sh[2][wid] = u2;
        sh[3][wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) t += sh[threadIdx.x][w];
        partials[blockIdx.x * 4 + threadIdx.x] = t;
    }
}

__global__ void reduce_final_kernel(const double *__restrict__ partials, int nblk, double *__restrict__ result)
{
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += partials[b * 4 + threadIdx.x];
        result[threadIdx.x] = t;
    }
}

cudaError_t launch_reduce(const double *macro, double *uprev, long long N, int update, double *partials, int nblk,
                          double *result, cudaStream_t s)
{
    reduce_partial_kernel<<<nblk, RED_THREADS, 0, s>>>(macro, uprev, N, update, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_kernel<<<1, 32, 0, s>>>(partials, nblk, result);
    return cudaGetLastError();
}

// ---- conversions (ref: optional [Q][ny] values subtracted before storing, in FP64) ----
template <typename Real, typename Store>
__global__ void to_store_kernel(const double *__restrict__ src, Store *__restrict__ dst, int Q, int nx, int ny, int pitch,
                                Real scale, const double *__restrict__ ref)
{
    const long long N = (long long)Q * nx * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / ((long long)nx * ny), r = i - q * nx * ny;
        const int y = int(r / nx), x = int(r - (long long)y * nx);
        Real v = Real(ref ? src[i] - ref[q * ny + y] : src[i]);
        if constexpr (scaled_<Store>()) v *= scale;
        st_(dst + (q * ny + y) * (long long)pitch + x, v);
    }
}
template <typename Real, typename Store>
__global__ void from_store_kernel(const Store *__restrict__ src, double *__restrict__ dst, int Q, int nx, int ny,
                                  int pitch, Real iscale, const double *__restrict__ ref)
{
    const long long N = (long long)Q * nx * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / ((long long)nx * ny), r = i - q * nx * ny;
        const int y = int(r / nx), x = int(r - (long long)y * nx);
        Real v = ld_<Real, Store>(src + (q * ny + y) * (long long)pitch + x);
        if constexpr (scaled_<Store>()) v *= iscale;
        dst[i] = ref ? double(v) + ref[q * ny + y] : double(v);
    }
}
template <typename Real, typename Store>
cudaError_t launch_to_store(const double *src, Store *dst, int Q, int nx, int ny, int pitch, Real scale,
                            const double *ref, cudaStream_t s)
{
    const long long N = (long long)Q * nx * ny;
    const int blocks = int((N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192);
    to_store_kernel<Real, Store><<<blocks, 256, 0, s>>>(src, dst, Q, nx, ny, pitch, scale, ref);
    return cudaGetLastError();
}
template <typename Real, typename Store>
cudaError_t launch_from_store(const Store *src, double *dst, int Q, int nx, int ny, int pitch, Real iscale,
                              const double *ref, cudaStream_t s)
{
    const long long N = (long long)Q * nx * ny;
    const int blocks = int((N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192);
    from_store_kernel<Real, Store><<<blocks, 256, 0, s>>>(src, dst, Q, nx, ny, pitch, iscale, ref);
    return cudaGetLastError();
}

__global__ void export_kernel(const double *__restrict__ src, void *dst, long long N, int to_float)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (to_float) ((float *)dst)[i] = float(src[i]);
        else ((double *)dst)[i] = src[i];
    }
}
cudaError_t launch_export(const double *src, void *dst, long long N, int to_float, cudaStream_t s)
{
    const int blocks = int((N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192);
    export_kernel<<<blocks, 256, 0, s>>>(src, dst, N, to_float);
    return cudaGetLastError();
}

#define LBM_INST_INIT(R, S, QF, QT) \
    template cudaError_t launch_init<R, S, QF, QT>(const StepArgs<R, S> &, double, double, int, cudaStream_t);
LBM_INST_INIT(double, double, 5, 5)
LBM_INST_INIT(double, double, 5, 9)
LBM_INST_INIT(double, double, 9, 5)
LBM_INST_INIT(double, double, 9, 9)
LBM_INST_INIT(float, float, 5, 5)
LBM_INST_INIT(float, float, 5, 9)
LBM_INST_INIT(float, float, 9, 5)
LBM_INST_INIT(float, float, 9, 9)
LBM_INST_INIT(float, __half, 5, 5)
LBM_INST_INIT(float, __half, 5, 9)
LBM_INST_INIT(float, __half, 9, 5)
LBM_INST_INIT(float, __half, 9, 9)
#undef LBM_INST_INIT

#define LBM_INST_CONV(R, S)                                                                                \
    template cudaError_t launch_to_store<R, S>(const double *, S *, int, int, int, int, R, const double *,        \
                                               cudaStream_t);                                                   \
    template cudaError_t launch_from_store<R, S>(const S *, double *, int, int, int, int, R, const double *,      \
                                                 cudaStream_t);
LBM_INST_CONV(double, double)
LBM_INST_CONV(float, float)
LBM_INST_CONV(float, __half)
#undef LBM_INST_CONV

}  // namespace lbm
