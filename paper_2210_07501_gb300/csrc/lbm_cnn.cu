// lbm_cnn.cu -- the learned warm start: a small convolutional surrogate that maps the
// channel's parameters and heating profile to its steady phi, u, v, T, with hand-written
// inference and training kernels (forward, backward-data, backward-weight, loss, Adam).
//
// Network: 6 layers of 3x3 convolutions, channels 12 -> 32 -> 32 -> 32 -> 32 -> 32 -> 4, SiLU
// between layers, none after the last.  Periodic in x (the channel is periodic), zero
// padding in y.  Weights, gradients and optimiser state are FP32; activations are stored in
// BF16 (or FP32, for gradient checks), every accumulation is FP32.  Layout NCHW.
// Deterministic: the weight gradients are summed in a fixed order (two passes).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <vector>

#include "../../include/lbm_gb300.h"

namespace {

constexpr int NL = 6;
constexpr int CH[NL + 1] = {12, 32, 32, 32, 32, 32, 4};
constexpr int TILE = 16;       // 16 x 16 output pixels per CTA
constexpr int CCH = 8;         // input channels staged per pass

template <typename A> __device__ __forceinline__ float to_f(A v)
{
    if constexpr (std::is_same<A, __nv_bfloat16>::value) return __bfloat162float(v);
    else return v;
}
template <typename A> __device__ __forceinline__ A from_f(float v)
{
    if constexpr (std::is_same<A, __nv_bfloat16>::value) return __float2bfloat16_rn(v);
    else return v;
}
__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// y[b][co][h][w] = bias[co] + sum_{ci, dy, dx} w[co][ci][dy][dx] * a[b][ci][h+dy-1][w+dx-1],
// a = x (layer 0) or silu(x) (later layers).
template <int CIN, int COUT, typename A>
__global__ void __launch_bounds__(TILE *TILE) conv_fwd(const A *__restrict__ x, const float *__restrict__ wgt,
                                                       const float *__restrict__ bias, A *__restrict__ y, int H, int W,
                                                       int act_in)
{
    __shared__ float s_x[CCH][TILE + 2][TILE + 2];
    __shared__ float s_w[COUT][CCH][9];
    const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
    const int w0 = blockIdx.x * TILE, h0 = blockIdx.y * TILE, b = blockIdx.z;
    const int wo = w0 + tx, ho = h0 + ty;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias[co];
    for (int c0 = 0; c0 < CIN; c0 += CCH) {
        const int nc = CIN - c0 < CCH ? CIN - c0 : CCH;
        for (int e = threadIdx.x; e < CCH * (TILE + 2) * (TILE + 2); e += TILE * TILE) {
            const int c = e / ((TILE + 2) * (TILE + 2)), r = e % ((TILE + 2) * (TILE + 2));
            const int iy = r / (TILE + 2), ix = r % (TILE + 2);
            const int hh = h0 + iy - 1, ww = (w0 + ix - 1 + W) % W;
            float v = 0.0f;
            if (c < nc && hh >= 0 && hh < H) {
                v = to_f(x[(((long long)b * CIN + c0 + c) * H + hh) * W + ww]);
                if (act_in) v = silu(v);
            }
            s_x[c][iy][ix] = v;
        }
        for (int e = threadIdx.x; e < COUT * CCH * 9; e += TILE * TILE) {
            const int co = e / (CCH * 9), r = e % (CCH * 9), c = r / 9, k = r % 9;
            s_w[co][c][k] = c < nc ? wgt[((co * CIN) + c0 + c) * 9 + k] : 0.0f;
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            float xv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) xv[k] = s_x[c][ty + k / 3][tx + k % 3];
#pragma unroll
            for (int co = 0; co < COUT; ++co) {
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k < 9; ++k) s += s_w[co][c][k] * xv[k];
                acc[co] += s;
            }
        }
        __syncthreads();
    }
    if (ho < H && wo < W)
#pragma unroll
        for (int co = 0; co < COUT; ++co) y[(((long long)b * COUT + co) * H + ho) * W + wo] = from_f<A>(acc[co]);
}

// da[b][ci][h][w] = sum_{co, dy, dx} w[co][ci][dy][dx] * dz[b][co][h-dy+1][w-dx+1]; then, for
// layers after the first, dz_in = da * silu'(z_in).
template <int CIN, int COUT, typename A>
__global__ void __launch_bounds__(TILE *TILE) conv_bwd_data(const float *__restrict__ dz, const float *__restrict__ wgt,
                                                            const A *__restrict__ zin, float *__restrict__ dzin, int H,
                                                            int W)
{
    __shared__ float s_d[CCH][TILE + 2][TILE + 2];
    __shared__ float s_w[CIN][CCH][9];
    const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
    const int w0 = blockIdx.x * TILE, h0 = blockIdx.y * TILE, b = blockIdx.z;
    const int wo = w0 + tx, ho = h0 + ty;
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.0f;
    for (int c0 = 0; c0 < COUT; c0 += CCH) {
        const int nc = COUT - c0 < CCH ? COUT - c0 : CCH;
        for (int e = threadIdx.x; e < CCH * (TILE + 2) * (TILE + 2); e += TILE * TILE) {
            const int c = e / ((TILE + 2) * (TILE + 2)), r = e % ((TILE + 2) * (TILE + 2));
            const int iy = r / (TILE + 2), ix = r % (TILE + 2);
            const int hh = h0 + iy - 1, ww = (w0 + ix - 1 + W) % W;
            float v = 0.0f;
            if (c < nc && hh >= 0 && hh < H) v = dz[(((long long)b * COUT + c0 + c) * H + hh) * W + ww];
            s_d[c][iy][ix] = v;
        }
        for (int e = threadIdx.x; e < CIN * CCH * 9; e += TILE * TILE) {
            const int ci = e / (CCH * 9), r = e % (CCH * 9), c = r / 9, k = r % 9;
            s_w[ci][c][k] = c < nc ? wgt[(((c0 + c) * CIN) + ci) * 9 + (8 - k)] : 0.0f;   // flipped kernel
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            float dv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) dv[k] = s_d[c][ty + k / 3][tx + k % 3];
#pragma unroll
            for (int ci = 0; ci < CIN; ++ci) {
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k < 9; ++k) s += s_w[ci][c][k] * dv[k];
                acc[ci] += s;
            }
        }
        __syncthreads();
    }
    if (ho < H && wo < W)
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) {
            const long long o = (((long long)b * CIN + ci) * H + ho) * W + wo;
            dzin[o] = acc[ci] * dsilu(to_f(zin[o]));
        }
}

// Partial weight and bias gradients of one 16 x 16 tile of one sample:
// part[tile][co][ci][k] = sum_p a[ci][p + k] dz[co][p],  part_b[tile][co] = sum_p dz[co][p].
template <int CIN, int COUT, typename A>
__global__ void __launch_bounds__(TILE *TILE) conv_bwd_weight(const A *__restrict__ x, const float *__restrict__ dz,
                                                              float *__restrict__ part, int H, int W, int act_in)
{
    extern __shared__ float smem[];
    float *s_x = smem;                                        // [CIN][TILE+2][TILE+2]
    float *s_d = smem + CIN * (TILE + 2) * (TILE + 2);        // [COUT][TILE][TILE]
    const int w0 = blockIdx.x * TILE, h0 = blockIdx.y * TILE, b = blockIdx.z;
    for (int e = threadIdx.x; e < CIN * (TILE + 2) * (TILE + 2); e += TILE * TILE) {
        const int c = e / ((TILE + 2) * (TILE + 2)), r = e % ((TILE + 2) * (TILE + 2));
        const int iy = r / (TILE + 2), ix = r % (TILE + 2);
        const int hh = h0 + iy - 1, ww = (w0 + ix - 1 + W) % W;
        float v = 0.0f;
        if (hh >= 0 && hh < H) {
            v = to_f(x[(((long long)b * CIN + c) * H + hh) * W + ww]);
            if (act_in) v = silu(v);
        }
        s_x[e] = v;
    }
    for (int e = threadIdx.x; e < COUT * TILE * TILE; e += TILE * TILE) {
        const int c = e / (TILE * TILE), r = e % (TILE * TILE), iy = r / TILE, ix = r % TILE;
        const int hh = h0 + iy, ww = w0 + ix;
        s_d[e] = (hh < H && ww < W) ? dz[(((long long)b * COUT + c) * H + hh) * W + ww] : 0.0f;
    }
    __syncthreads();
    const int nw = COUT * CIN * 9, tiles = gridDim.x * gridDim.y * gridDim.z;
    const int tile = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    for (int j = threadIdx.x; j < nw + COUT; j += TILE * TILE) {
        float s = 0.0f;
        if (j < nw) {
            const int co = j / (CIN * 9), r = j % (CIN * 9), ci = r / 9, k = r % 9, ky = k / 3, kx = k % 3;
            const float *xs = s_x + ci * (TILE + 2) * (TILE + 2);
            const float *ds = s_d + co * TILE * TILE;
            for (int py = 0; py < TILE; ++py)
#pragma unroll 4
                for (int px = 0; px < TILE; ++px) s += xs[(py + ky) * (TILE + 2) + px + kx] * ds[py * TILE + px];
        } else {
            const float *ds = s_d + (j - nw) * TILE * TILE;
            for (int p = 0; p < TILE * TILE; ++p) s += ds[p];
        }
        part[(long long)j * tiles + tile] = s;
    }
}

// grad[j] = sum over tiles of part[j][tile], in tile order.
__global__ void reduce_parts(const float *__restrict__ part, int tiles, int n, float *__restrict__ grad)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += part[(long long)j * tiles + t];
    grad[j] = (float)s;
}

// MSE loss on the last layer: dz = 2 (y - t) / N; per-block partial sums of (y - t)^2.
template <typename A>
__global__ void mse_grad(const A *__restrict__ y, const float *__restrict__ t, long long n, float *__restrict__ dz,
                         double *__restrict__ part)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = to_f(y[i]) - t[i];
        dz[i] = 2.0f * d / (float)n;
        s += (double)d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void adam_step(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                          float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <typename A> __global__ void to_act(const float *__restrict__ x, A *__restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = from_f<A>(x[i]);
}
template <typename A> __global__ void from_act(const A *__restrict__ x, float *__restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = to_f(x[i]);
}

int nparams_of_layer(int l) { return CH[l + 1] * CH[l] * 9 + CH[l + 1]; }

}  // namespace

struct lbm_cnn {
    int H = 0, W = 0, Bmax = 0, bf16 = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_params = 0;
    int off_w[NL], off_b[NL];
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // params, grads, Adam state
    void *act[NL + 1] = {nullptr};    // act[0] = input, act[l+1] = pre-activation output of layer l
    float *dz[2] = {nullptr, nullptr};
    float *part = nullptr;
    long long part_cap = 0;
    double *loss_part = nullptr, *loss_host = nullptr;
    int64_t t = 0;                    // Adam step
};

static thread_local char g_cnn_err[160] = "";

template <typename A> static cudaError_t cnn_forward_impl(lbm_cnn *c, int B)
{
    const dim3 grid((c->W + TILE - 1) / TILE, (c->H + TILE - 1) / TILE, B), blk(TILE * TILE);
    for (int l = 0; l < NL; ++l) {
        const A *x = (const A *)c->act[l];
        A *y = (A *)c->act[l + 1];
        const float *w = c->p + c->off_w[l], *bias = c->p + c->off_b[l];
        const int act_in = l > 0;
        if (l == 0) conv_fwd<CH[0], 32, A><<<grid, blk, 0, c->stream>>>(x, w, bias, y, c->H, c->W, act_in);
        else if (CH[l + 1] == 32) conv_fwd<32, 32, A><<<grid, blk, 0, c->stream>>>(x, w, bias, y, c->H, c->W, act_in);
        else conv_fwd<32, 4, A><<<grid, blk, 0, c->stream>>>(x, w, bias, y, c->H, c->W, act_in);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int CIN, int COUT, typename A>
static cudaError_t bwd_weight_launch(lbm_cnn *c, int l, int B, const float *dz)
{
    const dim3 grid((c->W + TILE - 1) / TILE, (c->H + TILE - 1) / TILE, B), blk(TILE * TILE);
    const size_t sm = (CIN * (TILE + 2) * (TILE + 2) + COUT * TILE * TILE) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(conv_bwd_weight<CIN, COUT, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    conv_bwd_weight<CIN, COUT, A><<<grid, blk, sm, c->stream>>>((const A *)c->act[l], dz, c->part, c->H, c->W, l > 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = nparams_of_layer(l), tiles = grid.x * grid.y * grid.z;
    // weights then biases: the layer's parameters are contiguous (w, then b)
    reduce_parts<<<(n + 255) / 256, 256, 0, c->stream>>>(c->part, tiles, n, c->g + c->off_w[l]);
    return cudaGetLastError();
}

template <typename A> static cudaError_t cnn_backward_impl(lbm_cnn *c, int B, const float *target, double *loss)
{
    const long long nout = (long long)B * CH[NL] * c->H * c->W;
    const int lb = 512;
    mse_grad<A><<<lb, 256, 0, c->stream>>>((const A *)c->act[NL], target, nout, c->dz[0], c->loss_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid((c->W + TILE - 1) / TILE, (c->H + TILE - 1) / TILE, B), blk(TILE * TILE);
    int cur = 0;
    for (int l = NL - 1; l >= 0; --l) {
        const float *dz = c->dz[cur];
        if (l == 0) e = bwd_weight_launch<CH[0], 32, A>(c, l, B, dz);
        else if (CH[l + 1] == 32) e = bwd_weight_launch<32, 32, A>(c, l, B, dz);
        else e = bwd_weight_launch<32, 4, A>(c, l, B, dz);
        if (e != cudaSuccess) return e;
        if (l > 0) {
            float *dzin = c->dz[1 - cur];
            const A *zin = (const A *)c->act[l];
            if (CH[l + 1] == 32) conv_bwd_data<32, 32, A><<<grid, blk, 0, c->stream>>>(dz, c->p + c->off_w[l], zin, dzin, c->H, c->W);
            else conv_bwd_data<32, 4, A><<<grid, blk, 0, c->stream>>>(dz, c->p + c->off_w[l], zin, dzin, c->H, c->W);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            cur = 1 - cur;
        }
    }
    e = cudaMemcpyAsync(c->loss_host, c->loss_part, lb * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    double s = 0.0;
    for (int i = 0; i < lb; ++i) s += c->loss_host[i];
    if (loss) *loss = s / (double)nout;
    return cudaSuccess;
}

static int cnn_fail(cudaError_t e, const char *what)
{
    snprintf(g_cnn_err, sizeof(g_cnn_err), "%s: %s", what, cudaGetErrorString(e));
    return LBM_ECUDA;
}

static cudaError_t cnn_load_input(lbm_cnn *c, const float *x, int B)
{
    const long long n = (long long)B * CH[0] * c->H * c->W;
    if (c->bf16) to_act<__nv_bfloat16><<<1024, 256, 0, c->stream>>>(x, (__nv_bfloat16 *)c->act[0], n);
    else to_act<float><<<1024, 256, 0, c->stream>>>(x, (float *)c->act[0], n);
    return cudaGetLastError();
}

extern "C" {

void lbm_cnn_destroy(lbm_cnn *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    float *fs[] = {c->p, c->g, c->m, c->v, c->dz[0], c->dz[1], c->part};
    for (float *f : fs)
        if (f) cudaFree(f);
    for (int l = 0; l <= NL; ++l)
        if (c->act[l]) cudaFree(c->act[l]);
    if (c->loss_part) cudaFree(c->loss_part);
    if (c->loss_host) cudaFreeHost(c->loss_host);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lbm_cnn_create(int32_t H, int32_t W, int32_t batch_max, int32_t bf16_activations, uint64_t seed, void *stream,
                   lbm_cnn **out)
{
    if (!out || H < 1 || W < 3 || batch_max < 1) return LBM_EINVAL;
    *out = nullptr;
    lbm_cnn *c = new (std::nothrow) lbm_cnn();
    if (!c) return LBM_ENOMEM;
    c->H = H;
    c->W = W;
    c->Bmax = batch_max;
    c->bf16 = bf16_activations ? 1 : 0;
    if (stream) c->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return LBM_ECUDA; }
        c->own_stream = true;
    }
    int off = 0;
    for (int l = 0; l < NL; ++l) {
        c->off_w[l] = off;
        off += CH[l + 1] * CH[l] * 9;
        c->off_b[l] = off;
        off += CH[l + 1];
    }
    c->n_params = off;
    const size_t asz = c->bf16 ? 2 : 4;
    const long long plane = (long long)H * W;
    bool ok = true;
    for (float **f : {&c->p, &c->g, &c->m, &c->v}) ok = ok && cudaMalloc((void **)f, off * sizeof(float)) == cudaSuccess;
    for (int l = 0; l <= NL && ok; ++l) ok = cudaMalloc(&c->act[l], (size_t)batch_max * CH[l] * plane * asz) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) ok = cudaMalloc((void **)&c->dz[k], (size_t)batch_max * 32 * plane * sizeof(float)) == cudaSuccess;
    const long long tiles = (long long)((W + TILE - 1) / TILE) * ((H + TILE - 1) / TILE) * batch_max;
    c->part_cap = tiles * (32 * 32 * 9 + 32);
    ok = ok && cudaMalloc((void **)&c->part, (size_t)c->part_cap * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&c->loss_part, 512 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&c->loss_host, 512 * sizeof(double)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); lbm_cnn_destroy(c); return LBM_ENOMEM; }
    // He-style initialisation from a 64-bit LCG (weights ~ U(-a, a), a = sqrt(6 / fan_in)), zero biases
    std::vector<float> h(off, 0.0f);
    uint64_t s = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    for (int l = 0; l < NL; ++l) {
        const float a = sqrtf(6.0f / (CH[l] * 9.0f)) * (l == NL - 1 ? 0.1f : 1.0f);
        for (int i = 0; i < CH[l + 1] * CH[l] * 9; ++i) {
            s = s * 6364136223846793005ULL + 1442695040888963407ULL;
            const double u01 = (double)(s >> 11) / 9007199254740992.0;
            h[c->off_w[l] + i] = (float)((2.0 * u01 - 1.0) * a);
        }
    }
    cudaError_t e = cudaMemcpy(c->p, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->m, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->v, 0, off * sizeof(float));
    if (e != cudaSuccess) { lbm_cnn_destroy(c); return LBM_ECUDA; }
    *out = c;
    return LBM_OK;
}

int lbm_cnn_num_params(const lbm_cnn *c, int64_t *n)
{
    if (!c || !n) return LBM_EINVAL;
    *n = c->n_params;
    return LBM_OK;
}

int lbm_cnn_get_params(lbm_cnn *c, float *host)
{
    if (!c || !host) return LBM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(host, c->p, c->n_params * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_fail(e, "lbm_cnn_get_params");
}

int lbm_cnn_set_params(lbm_cnn *c, const float *host)
{
    if (!c || !host) return LBM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(c->p, host, c->n_params * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->m, 0, c->n_params * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->v, 0, c->n_params * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->t = 0;
    return e == cudaSuccess ? LBM_OK : cnn_fail(e, "lbm_cnn_set_params");
}

int lbm_cnn_forward(lbm_cnn *c, const float *x, int32_t B, float *y)
{
    if (!c || !x || !y || B < 1 || B > c->Bmax) return LBM_EINVAL;
    cudaError_t e = cnn_load_input(c, x, B);
    if (e == cudaSuccess) e = c->bf16 ? cnn_forward_impl<__nv_bfloat16>(c, B) : cnn_forward_impl<float>(c, B);
    const long long n = (long long)B * CH[NL] * c->H * c->W;
    if (e == cudaSuccess) {
        if (c->bf16) from_act<__nv_bfloat16><<<1024, 256, 0, c->stream>>>((const __nv_bfloat16 *)c->act[NL], y, n);
        else from_act<float><<<1024, 256, 0, c->stream>>>((const float *)c->act[NL], y, n);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? LBM_OK : cnn_fail(e, "lbm_cnn_forward");
}

int lbm_cnn_gradients(lbm_cnn *c, const float *x, const float *target, int32_t B, float *grad_host, double *loss)
{
    if (!c || !x || !target || B < 1 || B > c->Bmax) return LBM_EINVAL;
    cudaError_t e = cnn_load_input(c, x, B);
    if (e == cudaSuccess) e = c->bf16 ? cnn_forward_impl<__nv_bfloat16>(c, B) : cnn_forward_impl<float>(c, B);
    if (e == cudaSuccess)
        e = c->bf16 ? cnn_backward_impl<__nv_bfloat16>(c, B, target, loss) : cnn_backward_impl<float>(c, B, target, loss);
    if (e == cudaSuccess && grad_host) {
        e = cudaMemcpyAsync(grad_host, c->g, c->n_params * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    return e == cudaSuccess ? LBM_OK : cnn_fail(e, "lbm_cnn_gradients");
}

int lbm_cnn_train_step(lbm_cnn *c, const float *x, const float *target, int32_t B, float lr, double *loss)
{
    int rc = lbm_cnn_gradients(c, x, target, B, nullptr, loss);
    if (rc) return rc;
    c->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)c->t), c2 = 1.0f - powf(b2, (float)c->t);
    adam_step<<<(c->n_params + 255) / 256, 256, 0, c->stream>>>(c->p, c->g, c->m, c->v, c->n_params, lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : cnn_fail(e, "lbm_cnn_train_step");
}

const char *lbm_cnn_strerror(void) { return g_cnn_err; }

}  // extern "C"
