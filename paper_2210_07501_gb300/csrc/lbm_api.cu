// lbm_api.cu -- host implementation of the C ABI declared in include/lbm_gb300.h.
//
// The handle owns two ping-pong copies of every population plane and of the stored
// pressure, the bottom-wall temperature table, the phase-field reference tables (the
// phase-field populations are stored as deviations from a flat reference interface), the
// macroscopic field buffer written by
// the last step of each lbm_step call (and at every residual check), the previous
// velocity for the residual, and the reduction scratch.  All work is queued on one CUDA
// stream; only the entry points that return data to the host synchronise it.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/lbm_gb300.h"
#include "lbm_internal.h"

using namespace lbm;

struct lbm_handle {
    lbm_domain dom;
    lbm_params prm;
    int prec, Qf, Qt, nx, ny, pitch;
    long long plane;        // ny * pitch
    size_t esize;           // bytes per stored population value
    size_t rsize;           // bytes per Real (pressure plane)
    cudaStream_t stream;
    bool own_stream;
    void *pop[2][3];        // [buffer][f, g, h]
    void *dp[2];
    void *twall;            // Real [3][nx]
    void *rtab;             // Real [RT_N][ny + 2]: phase-field reference row tables
    void *rowx;             // Real [ny][RX_N]: the same, grouped per output row
    double *phi0;           // [ny] reference phi profile
    double *fref;           // [Qf][ny] reference phase-field populations
    double *macro;          // [5][ny][nx]
    double *uprev;          // [2][ny][nx]
    double *partials;       // reduction scratch [nblk][4]
    double *result;         // [2][4]: last check, last diag; then the device fault word (8 bytes)
    double *host_result;    // pinned [9]
    double *staging;        // lazily allocated [9][ny][nx] doubles for state I/O
    int cur;
    int64_t step, check_interval, launches;
    int seg_rows;           // rows per CTA segment of the step kernel (0 = automatic)
    unsigned int tx_extra;  // lbm_test_stall_copies: extra bytes each copy stage waits for
    int64_t last_check_step, prev_check_step;
    bool have_check, have_prev_check;
    double res_du2, res_u2;
    double sf, sg, sh;
    Phys<double> P;
};

static thread_local char g_errbuf[256] = "";

static int cuda_fail(cudaError_t e, const char *what)
{
    snprintf(g_errbuf, sizeof(g_errbuf), "%s: %s", what, cudaGetErrorString(e));
    return LBM_ECUDA;
}
#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

template <typename Real> static Phys<Real> cast_phys(const Phys<double> &d)
{
    Phys<Real> p;
    p.W4 = Real(d.W4);
    p.csf = Real(d.csf);
    p.sigma0 = Real(d.sigma0);
    p.sigma1 = Real(d.sigma1);
    p.sigma2 = Real(d.sigma2);
    p.T_ref = Real(d.T_ref);
    p.dTcold = Real(d.dTcold);
    p.rhoA = Real(d.rhoA);
    p.drho = Real(d.drho);
    p.muA = Real(d.muA);
    p.dmu = Real(d.dmu);
    p.kA = Real(d.kA);
    p.dk = Real(d.dk);
    p.omega_phi = Real(d.omega_phi);
    p.Mphi = Real(d.Mphi);
    p.Fx = Real(d.Fx);
    p.Fy = Real(d.Fy);
    p.g2min = std::is_same<Real, double>::value ? Real(1e-24) : Real(1e-20);
    return p;
}

template <typename Real, typename Store> static StepArgs<Real, Store> make_args(const lbm_handle *h, int src, double *macro)
{
    StepArgs<Real, Store> A;
    A.nx = h->nx;
    A.ny = h->ny;
    A.pitch = h->pitch;
    A.plane = h->plane;
    const int dst = 1 - src;
    A.f_in = (const Store *)h->pop[src][0];
    A.g_in = (const Store *)h->pop[src][1];
    A.h_in = (const Store *)h->pop[src][2];
    A.f_out = (Store *)h->pop[dst][0];
    A.g_out = (Store *)h->pop[dst][1];
    A.h_out = (Store *)h->pop[dst][2];
    A.dp_in = (const Real *)h->dp[src];
    A.dp_out = (Real *)h->dp[dst];
    A.twall = (const Real *)h->twall;
    A.rtab = (const Real *)h->rtab;
    A.rowx = (const Real *)h->rowx;
    A.phi0 = h->phi0;
    A.fref = h->fref;
    A.macro = macro;
    for (int a = 0; a < 9; ++a) {
        const long long o = (long long)a * h->plane;
        A.fi[a] = A.f_in + (a < h->Qf ? o : 0);
        A.gi[a] = A.g_in + o;
        A.hi[a] = A.h_in + (a < h->Qt ? o : 0);
        A.fo[a] = A.f_out + (a < h->Qf ? o : 0);
        A.go[a] = A.g_out + o;
        A.ho[a] = A.h_out + (a < h->Qt ? o : 0);
    }
    A.P = cast_phys<Real>(h->P);
    A.sf = Real(h->sf);
    A.sg = Real(h->sg);
    A.sh = Real(h->sh);
    A.isf = Real(1.0 / h->sf);
    A.isg = Real(1.0 / h->sg);
    A.ish = Real(1.0 / h->sh);
    A.fault = (unsigned int *)(h->result + 8);
    A.tx_extra = h->tx_extra;
    return A;
}

// Dispatch a functor templated on <Real, Store, QF, QT> for the handle's configuration.
template <template <typename, typename, int, int> class Fn, typename... Args>
static cudaError_t dispatch(const lbm_handle *h, Args... args)
{
#define LBM_CASE(PREC, R, S)                                                          \
    if (h->prec == PREC) {                                                            \
        if (h->Qf == 5 && h->Qt == 5) return Fn<R, S, 5, 5>::run(h, args...);         \
        if (h->Qf == 5 && h->Qt == 9) return Fn<R, S, 5, 9>::run(h, args...);         \
        if (h->Qf == 9 && h->Qt == 5) return Fn<R, S, 9, 5>::run(h, args...);         \
        return Fn<R, S, 9, 9>::run(h, args...);                                       \
    }
    LBM_CASE(LBM_FP64, double, double)
    LBM_CASE(LBM_FP32, float, float)
    LBM_CASE(LBM_FP16, float, __half)
#undef LBM_CASE
    return cudaErrorInvalidValue;
}

template <typename R, typename S, int QF, int QT> struct StepFn {
    static cudaError_t run(const lbm_handle *h, int src, double *macro)
    {
        return launch_step<R, S, QF, QT>(make_args<R, S>(h, src, macro), h->stream, h->seg_rows);
    }
};
template <typename R, typename S, int QF, int QT> struct InitFn {
    static cudaError_t run(const lbm_handle *h, int dst, int defaults)
    {
        // init writes buffer `dst`: build args whose outputs are dst (inputs unused)
        StepArgs<R, S> A = make_args<R, S>(h, 1 - dst, h->macro);
        return launch_init<R, S, QF, QT>(A, h->dom.b, h->dom.W, defaults, h->stream);
    }
};

static size_t store_size(int prec) { return prec == LBM_FP64 ? 8 : (prec == LBM_FP32 ? 4 : 2); }
static size_t real_size(int prec) { return prec == LBM_FP64 ? 8 : 4; }

static void free_all(lbm_handle *h)
{
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 3; ++k)
            if (h->pop[b][k]) cudaFree(h->pop[b][k]);
        if (h->dp[b]) cudaFree(h->dp[b]);
    }
    if (h->twall) cudaFree(h->twall);
    if (h->rtab) cudaFree(h->rtab);
    if (h->rowx) cudaFree(h->rowx);
    if (h->phi0) cudaFree(h->phi0);
    if (h->fref) cudaFree(h->fref);
    if (h->macro) cudaFree(h->macro);
    if (h->uprev) cudaFree(h->uprev);
    if (h->partials) cudaFree(h->partials);
    if (h->result) cudaFree(h->result);
    if (h->staging) cudaFree(h->staging);
    if (h->host_result) cudaFreeHost(h->host_result);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

static int validate(const lbm_domain *d, const lbm_params *p)
{
    if (!d || !p) return LBM_EINVAL;
    if (d->nx < 3 || d->ny < 3) return LBM_EINVAL;
    // element offsets inside one population plane are 32-bit
    if ((long long)d->ny * (((long long)d->nx + 63) / 64 * 64) >= (1LL << 31)) return LBM_EINVAL;
    if ((d->q_phi != 5 && d->q_phi != 9) || (d->q_T != 5 && d->q_T != 9)) return LBM_EINVAL;
    if (d->precision < LBM_FP64 || d->precision > LBM_FP16 || d->heat_periods < 0) return LBM_EINVAL;
    if (!(d->W > 0.0) || !(d->b > 0.0) || !(d->b < d->ny)) return LBM_EINVAL;
    if (!(p->tau_flow > 0.5) || !(p->tau_T > 0.5) || !(p->tau_phi > 0.5)) return LBM_EINVAL;
    if (!(p->visc_ratio > 0.0) || !(p->cond_ratio > 0.0) || !(p->rho_bottom > 0.0) || !(p->rho_top > 0.0))
        return LBM_EINVAL;
    const double vals[] = {p->sigma0, p->sigma1, p->sigma2, p->T_ref, p->T_hot, p->T_cold, p->dT, p->Fx_ext, p->Fy_ext};
    for (double v : vals)
        if (!isfinite(v)) return LBM_EINVAL;
    return LBM_OK;
}

// Storage scale of the FP16 flow populations: g - w p0 carries w (dp + 3 rho c^2 e.u);
// scale the expected thermocapillary velocity (Marangoni stress balance, App. C) and the
// body-force velocity to O(0.1) so that they sit in FP16's normal range.
static double fp16_flow_scale(const lbm_domain *d, const lbm_params *p, double muA)
{
    const double dsig = fabs(p->sigma1) + 2.0 * fabs(p->sigma2) * (fabs(p->dT) + fabs(p->T_hot - p->T_ref));
    double u = dsig * fabs(p->dT) / muA * 0.25;
    u += (fabs(p->Fx_ext) + fabs(p->Fy_ext)) * (double)d->ny * d->ny / (8.0 * muA);
    u += fabs(p->sigma0) / (muA * (double)d->W) * 1e-3;
    if (!(u > 1e-12)) u = 1e-12;
    double s = exp2(floor(log2(0.05 / u)));
    if (s < 1.0) s = 1.0;
    if (s > 1073741824.0) s = 1073741824.0;
    return s;
}

// Compensated (Neumaier) summation: the sum of the terms rounded once, to within a unit in
// the last place of the result, however much the terms cancel.
struct KahanSum {
    double s = 0.0, c = 0.0;
    void add(double x)
    {
        const double t = s + x;
        c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

// Reference state of the phase-field lattice (Sec. 4.1): the flat tanh interface of width
// W at y = b, at rest, at its central-moment equilibrium with the normal pointing up,
//   k_ref(y) = (p, 0, M_phi theta(p), c^2 p, c^2 p, 0, 0, 0, c^4 p),  p = tanh profile,
//   r_a(y) = (P^-1 k_ref(y))_a  (u = 0: raw and central moments coincide).
// The kernels carry f - r.  The change of variables is exact for the FP64 numbers r_a(y)
// as they are, so every table is derived from those numbers: phi0(y) = sum_a r_a(y); the
// sum of the reference populations pulled into row y under the wall rules (specular
// reflection), R(y), enters as dR = R - phi0 = sum_a (r_a(pulled) - r_a(y)), summed with
// compensation so that it is exact to its own last place (dR feeds sum phi every step: a
// rounding error in it would add or remove phi each step); Ry(y) the first y moment of the
// pulled populations and t01(y) = sum_a e_ay r_a(y) give the first-moment constant
// c01 = (1 - omega) Ry + omega M_phi theta(phi0) - t01.  In FP32 dR is split into a high and
// a low part, and the parts are corrected to sum to zero over the rows.
static int build_phase_reference(lbm_handle *h)
{
    const int ny = h->ny, Q = h->Qf;
    const double b = h->dom.b, W = h->dom.W, M = h->P.Mphi, om = h->P.omega_phi, c2 = 1.0 / 3.0;
    std::vector<double> phi0(ny), r((size_t)Q * ny), tab((size_t)RT_N * (ny + 2), 0.0);
    for (int j = 0; j < ny; ++j) {
        const double y = j + 0.5;
        const double p = 0.5 + 0.5 * tanh(2.0 * (y - b) / W);
        const double t = M * 4.0 * p * (1.0 - p) / W;
        double k[9] = {p, 0.0, t, c2 * p, c2 * p, 0.0, 0.0, 0.0, c2 * c2 * p}, f[9];
        if (Q == 9) {
            f[0] = k[0] - k[3] - k[4] + k[8];
            f[1] = 0.5 * (k[1] + k[3] - k[7] - k[8]);
            f[2] = 0.5 * (k[2] + k[4] - k[6] - k[8]);
            f[3] = 0.5 * (-k[1] + k[3] + k[7] - k[8]);
            f[4] = 0.5 * (-k[2] + k[4] + k[6] - k[8]);
            f[5] = 0.25 * (k[5] + k[6] + k[7] + k[8]);
            f[6] = 0.25 * (-k[5] + k[6] - k[7] + k[8]);
            f[7] = 0.25 * (k[5] - k[6] - k[7] + k[8]);
            f[8] = 0.25 * (-k[5] - k[6] + k[7] + k[8]);
        } else {
            f[0] = k[0] - k[3] - k[4];
            f[1] = 0.5 * (k[1] + k[3]);
            f[2] = 0.5 * (k[2] + k[4]);
            f[3] = 0.5 * (k[3] - k[1]);
            f[4] = 0.5 * (k[4] - k[2]);
        }
        KahanSum s;
        for (int a = 0; a < Q; ++a) {
            r[(size_t)a * ny + j] = f[a];
            s.add(f[a]);
        }
        phi0[j] = s.value();
    }
    auto mirror = [ny](int y) {
        if (y < 0) y = -1 - y;
        if (y >= ny) y = 2 * ny - 1 - y;
        return y < 0 ? 0 : (y >= ny ? ny - 1 : y);
    };
    auto T = [&](int k, int row) -> double & { return tab[(size_t)k * (ny + 2) + row + 1]; };
    std::vector<double> dR(ny);
    for (int j = 0; j < ny; ++j) {
        KahanSum d, ry, t01;
        for (int a = 0; a < Q; ++a) {
            const int ey = ey_(a);
            const bool wall = (ey > 0 && j == 0) || (ey < 0 && j == ny - 1);
            const double v = wall ? r[(size_t)mir_(a) * ny + j] : r[(size_t)a * ny + (j - ey)];
            const double own = r[(size_t)a * ny + j];
            d.add(v);
            d.add(-own);
            ry.add(ey * v);
            t01.add(ey * own);
        }
        dR[j] = d.value();
        const double th0 = 4.0 * phi0[j] * (1.0 - phi0[j]) / W;
        T(RT_PHI0, j) = phi0[j];
        T(RT_TH0, j) = th0;
        T(RT_C01, j) = (1.0 - om) * ry.value() + om * M * th0 - t01.value();
    }
    for (int j = -1; j <= ny; ++j) T(RT_GREF, j) = 0.5 * (phi0[mirror(j + 1)] - phi0[mirror(j - 1)]);
    // dR in the kernels' precision as hi + lo, corrected so that the rows sum to zero
    int jmin = 0;
    KahanSum tot;
    for (int j = 0; j < ny; ++j) {
        const double hi = h->rsize == 8 ? dR[j] : (double)(float)dR[j];
        const double lo = h->rsize == 8 ? 0.0 : (double)(float)(dR[j] - hi);
        T(RT_DR, j) = hi;
        T(RT_DRLO, j) = lo;
        tot.add(hi);
        tot.add(lo);
        if (fabs(dR[j]) < fabs(dR[jmin])) jmin = j;
    }
    T(h->rsize == 8 ? RT_DR : RT_DRLO, jmin) -= tot.value();
    // per output row: the values the row-marching kernel stages with the row
    std::vector<double> rx((size_t)RX_N * ny, 0.0);
    for (int j = 0; j < ny; ++j) {
        double *o = rx.data() + (size_t)RX_N * j;
        o[RX_PHI0] = T(RT_PHI0, j);
        o[RX_TH0] = T(RT_TH0, j);
        o[RX_C01] = T(RT_C01, j);
        o[RX_GREF] = T(RT_GREF, j);
        o[RX_DR3] = T(RT_DR, mirror(j + 3));
        o[RX_DR3LO] = T(RT_DRLO, mirror(j + 3));
        o[RX_GREF1] = T(RT_GREF, j + 1);
    }
    cudaError_t e;
    if (h->rsize == 8) {
        e = cudaMemcpy(h->rtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->rowx, rx.data(), rx.size() * sizeof(double), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> tf(tab.size()), rf(rx.size());
        for (size_t i = 0; i < tab.size(); ++i) tf[i] = (float)tab[i];
        for (size_t i = 0; i < rx.size(); ++i) rf[i] = (float)rx[i];
        e = cudaMemcpy(h->rtab, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->rowx, rf.data(), rf.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(h->phi0, phi0.data(), ny * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->fref, r.data(), r.size() * sizeof(double), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "reference tables");
}

extern "C" {

const char *lbm_strerror(int status)
{
    switch (status) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return g_errbuf[0] ? g_errbuf : "CUDA error";
    case LBM_EUNSTABLE: return "non-finite value in the fields (unstable)";
    case LBM_ETIMEOUT: return "tolerance not reached within max_steps";
    case LBM_EIO: return "checkpoint I/O error";
    case LBM_EDEVICE: return "a step kernel gave up waiting for its copies (state invalid)";
    default: return "unknown status";
    }
}

static int reset_diag(lbm_handle *h)
{
    h->have_check = h->have_prev_check = false;
    h->last_check_step = h->prev_check_step = -1;
    h->res_du2 = h->res_u2 = 0.0;
    const size_t N = (size_t)h->nx * h->ny;
    CK(cudaMemsetAsync(h->uprev, 0, 2 * N * sizeof(double), h->stream));
    CK(cudaMemsetAsync(h->result + 8, 0, sizeof(double), h->stream));   // a new state clears a fault
    return LBM_OK;
}

int lbm_create(const lbm_domain *domain, const lbm_params *params, void *stream, lbm_handle **out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    int rc = validate(domain, params);
    if (rc) return rc;
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ENOMEM;
    h->dom = *domain;
    h->prm = *params;
    h->prec = domain->precision;
    h->Qf = domain->q_phi;
    h->Qt = domain->q_T;
    h->nx = domain->nx;
    h->ny = domain->ny;
    h->pitch = (domain->nx + 63) / 64 * 64;
    h->plane = (long long)h->ny * h->pitch;
    h->esize = store_size(h->prec);
    h->rsize = real_size(h->prec);
    h->check_interval = 100;
    cudaError_t e;
    if (stream) {
        h->stream = (cudaStream_t)stream;
        h->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaStreamCreate"); }
        h->own_stream = true;
    }
    const int Q[3] = {h->Qf, 9, h->Qt};
    const size_t N = (size_t)h->nx * h->ny;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        for (int k = 0; k < 3 && ok; ++k)
            ok = cudaMalloc(&h->pop[b][k], (size_t)Q[k] * h->plane * h->esize) == cudaSuccess;
        ok = ok && cudaMalloc(&h->dp[b], (size_t)h->plane * h->rsize) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&h->twall, 3 * (size_t)h->nx * h->rsize) == cudaSuccess;
    ok = ok && cudaMalloc(&h->rtab, (size_t)RT_N * (h->ny + 2) * h->rsize) == cudaSuccess;
    ok = ok && cudaMalloc(&h->rowx, (size_t)RX_N * h->ny * h->rsize) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&h->phi0, (size_t)h->ny * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&h->fref, (size_t)h->Qf * h->ny * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&h->macro, 5 * N * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&h->uprev, 2 * N * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&h->partials, (size_t)reduce_blocks() * 4 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&h->result, 9 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&h->host_result, 9 * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return LBM_ENOMEM;
    }
    cudaMemsetAsync(h->result, 0, 9 * sizeof(double), h->stream);
    h->host_result[8] = 0.0;
    // padding columns are never read, but keep them defined
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 3; ++k) cudaMemsetAsync(h->pop[b][k], 0, (size_t)Q[k] * h->plane * h->esize, h->stream);
        cudaMemsetAsync(h->dp[b], 0, (size_t)h->plane * h->rsize, h->stream);
    }
    // physical constants (Sec. 2-4), lattice units, c^2 = 1/3, c_p = 1
    const lbm_params *p = params;
    Phys<double> &P = h->P;
    P.W4 = 4.0 / domain->W;
    P.csf = 1.5 * domain->W;
    P.sigma0 = p->sigma0;
    P.sigma1 = p->sigma1;
    P.sigma2 = p->sigma2;
    P.T_ref = p->T_ref;
    P.dTcold = p->T_cold - p->T_ref;
    P.rhoA = p->rho_bottom;
    P.drho = p->rho_top - p->rho_bottom;
    const double nuA = (p->tau_flow - 0.5) / 3.0, alphaA = (p->tau_T - 0.5) / 3.0;
    P.muA = p->rho_bottom * nuA;
    P.dmu = (p->visc_ratio - 1.0) * P.muA;
    P.kA = p->rho_bottom * alphaA;
    P.dk = (p->cond_ratio - 1.0) * P.kA;
    P.omega_phi = 1.0 / p->tau_phi;
    P.Mphi = (1.0 / P.omega_phi - 0.5) / 3.0;
    P.Fx = p->Fx_ext;
    P.Fy = p->Fy_ext;
    P.g2min = 0.0;
    // FP16: the phase-field deviations f - r stay within [-1, 1]; 2^10 keeps them in the
    // normal range of FP16 down to ~6e-8
    h->sf = h->prec == LBM_FP16 ? 1024.0 : 1.0;
    h->sh = 1.0;
    h->sg = h->prec == LBM_FP16 ? fp16_flow_scale(domain, p, P.muA) : 1.0;
    rc = build_phase_reference(h);
    if (rc) { free_all(h); delete h; return rc; }
    // bottom-wall temperature minus T_ref at x - 1/2, x, x + 1/2 (heating peak at x = 0)
    {
        double *tw = (double *)malloc(3 * (size_t)h->nx * sizeof(double));
        if (!tw) { free_all(h); delete h; return LBM_ENOMEM; }
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < h->nx; ++i) {
                const double x = (double)i + 0.5 * (double)(k - 1);
                tw[k * h->nx + i] = p->T_hot + p->dT * cos(2.0 * M_PI * (double)domain->heat_periods * x / (double)h->nx) - p->T_ref;
            }
        cudaError_t ce;
        if (h->rsize == 8) {
            ce = cudaMemcpy(h->twall, tw, 3 * (size_t)h->nx * sizeof(double), cudaMemcpyHostToDevice);
        } else {
            float *twf = (float *)malloc(3 * (size_t)h->nx * sizeof(float));
            if (!twf) { free(tw); free_all(h); delete h; return LBM_ENOMEM; }
            for (int i = 0; i < 3 * h->nx; ++i) twf[i] = (float)tw[i];
            ce = cudaMemcpy(h->twall, twf, 3 * (size_t)h->nx * sizeof(float), cudaMemcpyHostToDevice);
            free(twf);
        }
        free(tw);
        if (ce != cudaSuccess) { free_all(h); delete h; return cuda_fail(ce, "cudaMemcpy(twall)"); }
    }
    rc = lbm_init_fields(h, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (rc) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return LBM_OK;
}

int lbm_init_fields(lbm_handle *h, const double *phi, const double *u, const double *v, const double *T,
                    const double *dp)
{
    if (!h) return LBM_EINVAL;
    const size_t N = (size_t)h->nx * h->ny;
    const double *src[5] = {phi, u, v, T, dp};
    int defaults = 0;
    for (int k = 0; k < 5; ++k) {
        if (src[k]) CK(cudaMemcpyAsync(h->macro + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        else defaults |= 1 << k;
    }
    h->cur = 0;
    CK(dispatch<InitFn>(h, 0, defaults));
    h->step = 0;
    int rc = reset_diag(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

static int run_check(lbm_handle *h)
{
    const long long N = (long long)h->nx * h->ny;
    CK(launch_reduce(h->macro, h->uprev, N, 1, h->partials, reduce_blocks(), h->result, h->stream));
    h->prev_check_step = h->last_check_step;
    h->have_prev_check = h->have_check;
    h->last_check_step = h->step;
    h->have_check = true;
    return LBM_OK;
}

int lbm_step(lbm_handle *h, int64_t nsteps)
{
    if (!h || nsteps < 0) return LBM_EINVAL;
    for (int64_t s = 0; s < nsteps; ++s) {
        const bool last = (s == nsteps - 1);
        const bool check = h->check_interval > 0 && ((h->step + 1) % h->check_interval == 0);
        double *macro = (last || check) ? h->macro : nullptr;
        CK(dispatch<StepFn>(h, h->cur, macro));
        h->cur = 1 - h->cur;
        h->step += 1;
        h->launches += 1;
        if (check) {
            int rc = run_check(h);
            if (rc) return rc;
        }
    }
    return LBM_OK;
}

int lbm_fields(lbm_handle *h, double *phi, double *u, double *v, double *T, double *dp)
{
    if (!h) return LBM_EINVAL;
    const size_t N = (size_t)h->nx * h->ny;
    double *dst[5] = {phi, u, v, T, dp};
    for (int k = 0; k < 5; ++k)
        if (dst[k]) CK(cudaMemcpyAsync(dst[k], h->macro + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->host_result + 8, h->result + 8, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (*(const unsigned int *)(h->host_result + 8)) return LBM_EDEVICE;
    return LBM_OK;
}

int lbm_fields_device(lbm_handle *h, void *phi, void *u, void *v, void *T, void *dp, int dtype)
{
    if (!h || (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32)) return LBM_EINVAL;
    const long long N = (long long)h->nx * h->ny;
    void *dst[5] = {phi, u, v, T, dp};
    for (int k = 0; k < 5; ++k)
        if (dst[k]) CK(launch_export(h->macro + k * N, dst[k], N, dtype == LBM_DTYPE_F32, h->stream));
    return LBM_OK;
}

int lbm_diag(lbm_handle *h, double *mass, double *residual, int64_t *step)
{
    if (!h) return LBM_EINVAL;
    const long long N = (long long)h->nx * h->ny;
    // residual terms of the last check, then a fresh mass / finiteness reduction
    CK(cudaMemcpyAsync(h->host_result, h->result, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(launch_reduce(h->macro, h->uprev, N, 0, h->partials, reduce_blocks(), h->result + 4, h->stream));
    CK(cudaMemcpyAsync(h->host_result + 4, h->result + 4, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const double *r = h->host_result;
    if (*(const unsigned int *)(r + 8)) return LBM_EDEVICE;
    if (mass) *mass = r[4];
    if (residual) {
        const int64_t K = h->last_check_step - h->prev_check_step;
        if (h->have_check && h->have_prev_check && K > 0 && r[2] > 0.0)
            *residual = sqrt(r[1]) / ((double)K * sqrt(r[2]));
        else
            *residual = -1.0;
    }
    if (step) *step = h->step;
    if (r[7] > 0.0 || (h->have_check && r[3] > 0.0)) return LBM_EUNSTABLE;
    return LBM_OK;
}

int lbm_set_check_interval(lbm_handle *h, int32_t K)
{
    if (!h || K < 1) return LBM_EINVAL;
    h->check_interval = K;
    return LBM_OK;
}

int lbm_run_to_steady(lbm_handle *h, double tol, int64_t max_steps, int64_t *steps_taken)
{
    if (!h || !(tol > 0.0) || max_steps < 0) return LBM_EINVAL;
    int64_t done = 0;
    int rc = LBM_ETIMEOUT;
    while (done < max_steps) {
        int64_t n = h->check_interval - (h->step % h->check_interval);
        if (n > max_steps - done) n = max_steps - done;
        int e = lbm_step(h, n);
        if (e) return e;
        done += n;
        double res;
        e = lbm_diag(h, nullptr, &res, nullptr);
        if (e) { rc = e; break; }
        if (h->last_check_step == h->step && res >= 0.0 && res <= tol) { rc = LBM_OK; break; }
    }
    if (steps_taken) *steps_taken = done;
    return rc;
}

}  // extern "C"

template <typename R, typename S, int QF, int QT> struct AutoSegFn {
    static cudaError_t run(const lbm_handle *h, int *rows)
    {
        *rows = auto_segment<R, S, QF, QT>(h->nx, h->ny);
        return cudaGetLastError();
    }
};

template <typename R, typename S, int QF, int QT> struct GetFn {
    static cudaError_t run(const lbm_handle *h, double *stage, int lattice, int Q, int toStore)
    {
        const double sc = lattice == 0 ? h->sf : (lattice == 1 ? h->sg : h->sh);
        const double *ref = lattice == 0 ? h->fref : nullptr;   // phase field: f - r stored
        if (toStore)
            return launch_to_store<R, S>(stage, (S *)h->pop[h->cur][lattice], Q, h->nx, h->ny, h->pitch, R(sc), ref,
                                         h->stream);
        return launch_from_store<R, S>((const S *)h->pop[h->cur][lattice], stage, Q, h->nx, h->ny, h->pitch,
                                       R(1.0 / sc), ref, h->stream);
    }
};
template <typename R, typename S, int QF, int QT> struct DpFn {
    static cudaError_t run(const lbm_handle *h, double *stage, int toStore)
    {
        if (toStore)
            return launch_to_store<R, R>(stage, (R *)h->dp[h->cur], 1, h->nx, h->ny, h->pitch, R(1), nullptr, h->stream);
        return launch_from_store<R, R>((const R *)h->dp[h->cur], stage, 1, h->nx, h->ny, h->pitch, R(1), nullptr,
                                       h->stream);
    }
};

extern "C" {

static int ensure_staging(lbm_handle *h)
{
    if (h->staging) return LBM_OK;
    const size_t N = (size_t)h->nx * h->ny;
    if (cudaMalloc((void **)&h->staging, 9 * N * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ENOMEM;
    }
    return LBM_OK;
}

int lbm_get_state(lbm_handle *h, double *f, double *g, double *hT, double *dp)
{
    if (!h || !f || !g || !hT || !dp) return LBM_EINVAL;
    int rc = ensure_staging(h);
    if (rc) return rc;
    const size_t N = (size_t)h->nx * h->ny;
    double *dst[3] = {f, g, hT};
    const int Q[3] = {h->Qf, 9, h->Qt};
    for (int k = 0; k < 3; ++k) {
        CK(dispatch<GetFn>(h, h->staging, k, Q[k], 0));
        CK(cudaMemcpyAsync(dst[k], h->staging, Q[k] * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    CK(dispatch<DpFn>(h, h->staging, 0));
    CK(cudaMemcpyAsync(dp, h->staging, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_state(lbm_handle *h, const double *f, const double *g, const double *hT, const double *dp)
{
    if (!h || !f || !g || !hT || !dp) return LBM_EINVAL;
    int rc = ensure_staging(h);
    if (rc) return rc;
    const size_t N = (size_t)h->nx * h->ny;
    const double *src[3] = {f, g, hT};
    const int Q[3] = {h->Qf, 9, h->Qt};
    for (int k = 0; k < 3; ++k) {
        CK(cudaMemcpyAsync(h->staging, src[k], Q[k] * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(dispatch<GetFn>(h, h->staging, k, Q[k], 1));
    }
    CK(cudaMemcpyAsync(h->staging, dp, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(dispatch<DpFn>(h, h->staging, 1));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// ---- checkpoints ----
static uint32_t crc32_update(uint32_t crc, const unsigned char *p, size_t n)
{
    static uint32_t table[256];
    static bool init = false;
    if (!init) {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : (c >> 1);
            table[i] = c;
        }
        init = true;
    }
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

struct ckpt_header {
    char magic[8];
    uint32_t version, crc;
    int64_t step;
    lbm_domain dom;
    lbm_params prm;
    uint64_t payload;
};

static size_t state_bytes(const lbm_handle *h)
{
    return ((size_t)(h->Qf + 9 + h->Qt) * h->plane) * h->esize + (size_t)h->plane * h->rsize;
}

int lbm_save(lbm_handle *h, const char *path)
{
    if (!h || !path) return LBM_EINVAL;
    const size_t bytes = state_bytes(h);
    unsigned char *buf = (unsigned char *)malloc(bytes);
    if (!buf) return LBM_ENOMEM;
    size_t off = 0;
    const int Q[3] = {h->Qf, 9, h->Qt};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        const size_t nb = (size_t)Q[k] * h->plane * h->esize;
        e = cudaMemcpyAsync(buf + off, h->pop[h->cur][k], nb, cudaMemcpyDeviceToHost, h->stream);
        off += nb;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + off, h->dp[h->cur], (size_t)h->plane * h->rsize, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { free(buf); return cuda_fail(e, "lbm_save copy"); }
    ckpt_header hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "LBMGB300", 8);
    hd.version = 2;
    hd.step = h->step;
    hd.dom = h->dom;
    hd.prm = h->prm;
    hd.payload = bytes;
    hd.crc = crc32_update(0, buf, bytes);
    FILE *fp = fopen(path, "wb");
    int rc = LBM_OK;
    if (!fp) rc = LBM_EIO;
    else {
        if (fwrite(&hd, sizeof(hd), 1, fp) != 1 || fwrite(buf, 1, bytes, fp) != bytes) rc = LBM_EIO;
        if (fclose(fp) != 0) rc = LBM_EIO;
    }
    free(buf);
    return rc;
}

int lbm_load(lbm_handle *h, const char *path)
{
    if (!h || !path) return LBM_EINVAL;
    FILE *fp = fopen(path, "rb");
    if (!fp) return LBM_EIO;
    ckpt_header hd;
    const size_t bytes = state_bytes(h);
    // the stored phase-field deviations are relative to a reference set by b, W and M_phi
    if (fread(&hd, sizeof(hd), 1, fp) != 1 || memcmp(hd.magic, "LBMGB300", 8) != 0 || hd.version != 2 ||
        hd.payload != bytes || hd.dom.nx != h->dom.nx || hd.dom.ny != h->dom.ny || hd.dom.q_phi != h->dom.q_phi ||
        hd.dom.q_T != h->dom.q_T || hd.dom.precision != h->dom.precision || hd.dom.b != h->dom.b ||
        hd.dom.W != h->dom.W || hd.prm.tau_phi != h->prm.tau_phi) {
        fclose(fp);
        return LBM_EIO;
    }
    unsigned char *buf = (unsigned char *)malloc(bytes);
    if (!buf) { fclose(fp); return LBM_ENOMEM; }
    const bool ok = fread(buf, 1, bytes, fp) == bytes;
    fclose(fp);
    if (!ok || crc32_update(0, buf, bytes) != hd.crc) { free(buf); return LBM_EIO; }
    size_t off = 0;
    const int Q[3] = {h->Qf, 9, h->Qt};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        const size_t nb = (size_t)Q[k] * h->plane * h->esize;
        e = cudaMemcpyAsync(h->pop[h->cur][k], buf + off, nb, cudaMemcpyHostToDevice, h->stream);
        off += nb;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dp[h->cur], buf + off, (size_t)h->plane * h->rsize, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    free(buf);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_load copy");
    h->step = hd.step;
    return reset_diag(h);
}

int lbm_set_segment(lbm_handle *h, int32_t rows)
{
    if (!h || rows < 0) return LBM_EINVAL;
    h->seg_rows = rows;
    return LBM_OK;
}

int lbm_test_stall_copies(lbm_handle *h, int32_t on)
{
    if (!h) return LBM_EINVAL;
    h->tx_extra = on ? 16u : 0u;
    return LBM_OK;
}

int lbm_autotune(lbm_handle *h, int32_t reps, int32_t *rows)
{
    if (!h || reps < 1) return LBM_EINVAL;
    // candidates: the automatic choice (whole waves), then fixed segment lengths up to the
    // channel height
    int cand[16], nc = 0;
    int autoseg = 0;
    CK(dispatch<AutoSegFn>(h, &autoseg));
    cand[nc++] = autoseg;
    const int fixed[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256};
    for (int f : fixed)
        if (f < h->ny && f != autoseg && nc < 16) cand[nc++] = f;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int saved = h->seg_rows;
    float best_ms = 1e30f;
    int best = 0;
    int rc = LBM_OK;
    for (int k = 0; k < nc && rc == LBM_OK; ++k) {
        h->seg_rows = cand[k];
        // the kernel reads buffer cur and writes the other one; launching it again from
        // the same buffer leaves the state and the step count untouched
        cudaError_t e = dispatch<StepFn>(h, h->cur, (double *)nullptr);      // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = dispatch<StepFn>(h, h->cur, (double *)nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { rc = cuda_fail(e, "lbm_autotune"); break; }
        if (ms < best_ms) { best_ms = ms; best = cand[k]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->seg_rows = rc == LBM_OK ? best : saved;
    if (rows) *rows = h->seg_rows;
    return rc;
}

int lbm_bytes_per_node(const lbm_handle *h, int64_t *bytes)
{
    if (!h || !bytes) return LBM_EINVAL;
    *bytes = (int64_t)(2 * (h->Qf + 9 + h->Qt) * h->esize + 2 * h->rsize);
    return LBM_OK;
}

int lbm_launch_count(const lbm_handle *h, int64_t *launches)
{
    if (!h || !launches) return LBM_EINVAL;
    *launches = h->launches;
    return LBM_OK;
}

void lbm_destroy(lbm_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"

// ======================================================================================
// Batched sweep: many channels of uneven size stepped by one kernel launch per step.
// ======================================================================================

struct lbm_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<lbm_handle *> h;       // per-case state (allocated on the batch stream)
    void *d_args[2] = {nullptr, nullptr};   // StepArgs per case, source buffer 0 / 1, no macros
    void *d_args_m[2] = {nullptr, nullptr}; // same, writing the macroscopic fields
    int4 *d_ctas = nullptr;
    int n_ctas = 0, seg = 32;
    int *d_active = nullptr;
    std::vector<int> active;
    double *d_results = nullptr;       // [n][4] reduction results of the last check, then the fault word
    double *h_results = nullptr;       // pinned copy
    std::vector<int64_t> steps;        // steps taken per case
    std::vector<double> residual;      // last residual per case (-1 before two checks)
    std::vector<int> checks;
    int64_t K = 100;                   // steps per chunk (even), one residual check per chunk
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
};

template <typename R, typename S, int QF, int QT> struct BatchArgsFn {
    static cudaError_t run(const lbm_handle *, lbm_batch *b)
    {
        const size_t sz = sizeof(StepArgs<R, S>);
        std::vector<StepArgs<R, S>> a(b->n);
        for (int par = 0; par < 2; ++par)
            for (int m = 0; m < 2; ++m) {
                for (int c = 0; c < b->n; ++c) {
                    a[c] = make_args<R, S>(b->h[c], par, m ? b->h[c]->macro : nullptr);
                    a[c].fault = (unsigned int *)(b->d_results + 4 * (size_t)b->n);   // one word per batch
                }
                void *&dst = m ? b->d_args_m[par] : b->d_args[par];
                if (!dst) {
                    cudaError_t e = cudaMalloc(&dst, sz * b->n);
                    if (e != cudaSuccess) return e;
                }
                cudaError_t e = cudaMemcpy(dst, a.data(), sz * b->n, cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return e;
            }
        return cudaSuccess;
    }
};

template <typename R, typename S, int QF, int QT> struct BatchTableFn {
    static cudaError_t run(const lbm_handle *, lbm_batch *b, int seg)
    {
        const int TX = step_strip_width<R, S, QF, QT>();
        std::vector<int4> t;
        for (int c = 0; c < b->n; ++c) {
            const int strips = (b->h[c]->nx + TX - 1) / TX, segs = (b->h[c]->ny + seg - 1) / seg;
            for (int by = 0; by < segs; ++by)
                for (int bx = 0; bx < strips; ++bx) t.push_back(make_int4(c, bx, by, 0));
        }
        if (b->d_ctas) cudaFree(b->d_ctas);
        b->d_ctas = nullptr;
        cudaError_t e = cudaMalloc((void **)&b->d_ctas, t.size() * sizeof(int4));
        if (e != cudaSuccess) return e;
        b->n_ctas = (int)t.size();
        b->seg = seg;
        return cudaMemcpy(b->d_ctas, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
};

template <typename R, typename S, int QF, int QT> struct BatchStepFn {
    static cudaError_t run(const lbm_handle *, lbm_batch *b, int par, int macro)
    {
        const StepArgs<R, S> *args = (const StepArgs<R, S> *)(macro ? b->d_args_m[par] : b->d_args[par]);
        return launch_batch<R, S, QF, QT>(args, b->d_ctas, b->n_ctas, b->d_active, b->seg, b->stream);
    }
};

template <typename R, typename S, int QF, int QT> struct BatchSlotsFn {
    static cudaError_t run(const lbm_handle *, int *slots)
    {
        *slots = resident_ctas<R, S, QF, QT>();
        return cudaSuccess;
    }
};

static int batch_capture(lbm_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_valid = false;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int64_t k = 0; k < b->K && e == cudaSuccess; ++k)
        e = dispatch<BatchStepFn>(b->h[0], b, (int)(k & 1), (int)(k == b->K - 1));
    for (int c = 0; c < b->n && e == cudaSuccess; ++c) {
        lbm_handle *h = b->h[c];
        e = launch_reduce(h->macro, h->uprev, (long long)h->nx * h->ny, 1, h->partials, reduce_blocks(),
                          b->d_results + 4 * c, b->stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "batch capture"); }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    b->graph_valid = true;
    return LBM_OK;
}

extern "C" {

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (int p = 0; p < 2; ++p) {
        if (b->d_args[p]) cudaFree(b->d_args[p]);
        if (b->d_args_m[p]) cudaFree(b->d_args_m[p]);
    }
    if (b->d_ctas) cudaFree(b->d_ctas);
    if (b->d_active) cudaFree(b->d_active);
    if (b->d_results) cudaFree(b->d_results);
    if (b->h_results) cudaFreeHost(b->h_results);
    for (lbm_handle *h : b->h) lbm_destroy(h);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int lbm_batch_create(int32_t n, const lbm_domain *domains, const lbm_params *params, void *stream, lbm_batch **out)
{
    if (!out || n < 1 || !domains || !params) return LBM_EINVAL;
    *out = nullptr;
    for (int c = 0; c < n; ++c) {
        int rc = validate(&domains[c], &params[c]);
        if (rc) return rc;
        if (domains[c].precision != domains[0].precision || domains[c].q_phi != domains[0].q_phi ||
            domains[c].q_T != domains[0].q_T)
            return LBM_EINVAL;
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    b->n = n;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
        b->own_stream = true;
    }
    for (int c = 0; c < n; ++c) {
        lbm_handle *h = nullptr;
        int rc = lbm_create(&domains[c], &params[c], (void *)b->stream, &h);
        if (rc) { lbm_batch_destroy(b); return rc; }
        b->h.push_back(h);
    }
    b->active.assign(n, 1);
    b->steps.assign(n, 0);
    b->residual.assign(n, -1.0);
    b->checks.assign(n, 0);
    bool ok = cudaMalloc((void **)&b->d_active, n * sizeof(int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_results, (4 * (size_t)n + 1) * sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void **)&b->h_results, (4 * (size_t)n + 1) * sizeof(double)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); lbm_batch_destroy(b); return LBM_ENOMEM; }
    cudaError_t e = cudaMemcpy(b->d_active, b->active.data(), n * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_results, 0, (4 * (size_t)n + 1) * sizeof(double));
    if (e == cudaSuccess) e = dispatch<BatchArgsFn>(b->h[0], b);
    int slots = 0;
    if (e == cudaSuccess) e = dispatch<BatchSlotsFn>(b->h[0], &slots);
    if (e == cudaSuccess) e = dispatch<BatchTableFn>(b->h[0], b, 32);
    if (e != cudaSuccess) { int rc = cuda_fail(e, "lbm_batch_create"); lbm_batch_destroy(b); return rc; }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_check_interval(lbm_batch *b, int32_t K)
{
    if (!b || K < 2 || (K & 1)) return LBM_EINVAL;
    b->K = K;
    b->graph_valid = false;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch *b, int32_t reps, int32_t *rows)
{
    if (!b || reps < 1) return LBM_EINVAL;
    int maxny = 0;
    for (lbm_handle *h : b->h) maxny = h->ny > maxny ? h->ny : maxny;
    const int cand[] = {8, 12, 16, 24, 32, 48, 64, 96, 128};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = b->seg, rc = LBM_OK;
    for (int seg : cand) {
        if (seg > maxny && seg != cand[0]) continue;
        cudaError_t e = dispatch<BatchTableFn>(b->h[0], b, seg);
        // launches from buffer 0 into buffer 1 leave the state (in buffer 0) untouched
        if (e == cudaSuccess) e = dispatch<BatchStepFn>(b->h[0], b, 0, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = dispatch<BatchStepFn>(b->h[0], b, 0, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { rc = cuda_fail(e, "lbm_batch_autotune"); break; }
        if (ms < best_ms) { best_ms = ms; best = seg; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == LBM_OK) {
        cudaError_t e = dispatch<BatchTableFn>(b->h[0], b, best);
        if (e != cudaSuccess) rc = cuda_fail(e, "lbm_batch_autotune");
    }
    b->graph_valid = false;
    if (rows) *rows = b->seg;
    return rc;
}

int lbm_batch_step(lbm_batch *b, int64_t nsteps)
{
    if (!b || nsteps < 0 || nsteps % b->K) return LBM_EINVAL;
    if (!b->graph_valid) {
        int rc = batch_capture(b);
        if (rc) return rc;
    }
    for (int64_t done = 0; done < nsteps; done += b->K) {
        CK(cudaGraphLaunch(b->graph, b->stream));
        CK(cudaMemcpyAsync(b->h_results, b->d_results, (4 * (size_t)b->n + 1) * sizeof(double),
                           cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        if (*(const unsigned int *)(b->h_results + 4 * (size_t)b->n)) return LBM_EDEVICE;
        for (int c = 0; c < b->n; ++c) {
            if (!b->active[c]) continue;
            lbm_handle *h = b->h[c];
            h->step += b->K;
            h->launches += b->K;
            b->steps[c] += b->K;
            b->checks[c] += 1;
            const double *r = b->h_results + 4 * c;
            b->residual[c] = (b->checks[c] >= 2 && r[2] > 0.0) ? sqrt(r[1]) / ((double)b->K * sqrt(r[2])) : -1.0;
            if (r[3] > 0.0) return LBM_EUNSTABLE;
        }
    }
    return LBM_OK;
}

int lbm_batch_run_to_steady(lbm_batch *b, double tol, int64_t max_steps, int64_t *steps, int32_t *converged)
{
    if (!b || !(tol > 0.0) || max_steps < 0) return LBM_EINVAL;
    int rc = LBM_OK;
    int64_t done = 0;
    for (;;) {
        int n_active = 0;
        for (int c = 0; c < b->n; ++c) n_active += b->active[c];
        if (n_active == 0 || done + b->K > max_steps) break;
        rc = lbm_batch_step(b, b->K);
        if (rc) break;
        done += b->K;
        bool changed = false;
        for (int c = 0; c < b->n; ++c)
            if (b->active[c] && b->residual[c] >= 0.0 && b->residual[c] <= tol) {
                b->active[c] = 0;
                changed = true;
            }
        if (changed) CK(cudaMemcpyAsync(b->d_active, b->active.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    }
    bool all = true;
    for (int c = 0; c < b->n; ++c) {
        const bool conv = b->residual[c] >= 0.0 && b->residual[c] <= tol;
        if (steps) steps[c] = b->steps[c];
        if (converged) converged[c] = conv ? 1 : 0;
        all = all && conv;
    }
    if (rc) return rc;
    return all ? LBM_OK : LBM_ETIMEOUT;
}

int lbm_batch_fields(lbm_batch *b, int32_t c, double *phi, double *u, double *v, double *T, double *dp)
{
    if (!b || c < 0 || c >= b->n) return LBM_EINVAL;
    return lbm_fields(b->h[c], phi, u, v, T, dp);
}

int lbm_batch_diag(lbm_batch *b, int32_t c, double *residual, int64_t *steps)
{
    if (!b || c < 0 || c >= b->n) return LBM_EINVAL;
    if (residual) *residual = b->residual[c];
    if (steps) *steps = b->steps[c];
    return LBM_OK;
}

int lbm_batch_init_fields(lbm_batch *b, int32_t c, const double *phi, const double *u, const double *v,
                          const double *T, const double *dp)
{
    if (!b || c < 0 || c >= b->n) return LBM_EINVAL;
    int rc = lbm_init_fields(b->h[c], phi, u, v, T, dp);
    if (rc) return rc;
    b->steps[c] = 0;
    b->residual[c] = -1.0;
    b->checks[c] = 0;
    b->active[c] = 1;
    CK(cudaMemcpyAsync(b->d_active, b->active.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_size(const lbm_batch *b, int32_t *n, int32_t *ctas, int32_t *rows)
{
    if (!b) return LBM_EINVAL;
    if (n) *n = b->n;
    if (ctas) *ctas = b->n_ctas;
    if (rows) *rows = b->seg;
    return LBM_OK;
}

}  // extern "C"
