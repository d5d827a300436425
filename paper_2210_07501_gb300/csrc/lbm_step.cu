// lbm_step.cu -- the fused time step of the coupled three-lattice central-moment LB
// method (arXiv 2210.07501, Sec. 4.1-4.3) for sm_103a.
//
// Per step and node: pull f and h (Sec. 4.1, 4.3 streaming with the Sec. 5.1 wall rules)
// and form phi = sum f and T - T_ref = sum h; stage phi (radius 2), sigma(T) - sigma0 and
// p^{n-1} - p0 (radius 1) in shared memory (ghost rows: phi, p mirrored; T = 2 T_w - T_adj);
// form the unit normal n = grad phi / |grad phi|; then the curvature term div n, grad sigma,
// grad p, the CSF force with delta_s = 1.5 W |grad phi|^2 (Sec. 3), the pressure force
// F_p = -grad(p - rho c^2) with the stored p of the previous step, pull g, form u and p
// (Sec. 4.2), collide all three lattices in central-moment space and write the
// post-collision populations and p to the other buffer.
// Populations live in SoA planes [Q][ny][pitch], x fastest: every pull of a warp is a
// contiguous (shifted) row segment.  No tensor cores: the step is a bandwidth-bound stencil.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

// ---- row-marching sliding window ------------------------------------------------------
// One CTA of TX threads owns a TX-column strip and walks up a segment of rows.  Shared
// memory holds rings of the last rows: phi (8 rows, radius-2 halo columns), the pair
// (sigma - sigma0, p - p0) and the unit normal (4 rows, radius-1 halo columns).  For output
// row y the CTA adds phi of row y + 2 (from f pulled there, kept in registers until row y
// collides), sigma and p of row y + 1 (from h pulled there, kept one row), the normals of
// row y + 1, and then collides row y.  The loads for the next row are issued before the
// current row's barriers and collisions (one-row software pipeline).  Every thread works
// on the same row, so wall tests and row addresses are uniform across the CTA; only 4 halo
// columns per strip are recomputed.
template <typename Real> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

template <typename Real>
__device__ __forceinline__ void grad3_(const Real *rm, const Real *r0, const Real *rp, int c, Real &gx, Real &gy)
{
    const Real c1 = Real(1.0 / 3.0), c2 = Real(1.0 / 12.0);
    const Real ne = rp[c + 1], nw = rp[c - 1], se = rm[c + 1], sw = rm[c - 1];
    gx = c1 * (r0[c + 1] - r0[c - 1]) + c2 * ((ne - nw) + (se - sw));
    gy = c1 * (rp[c] - rm[c]) + c2 * ((ne - se) + (nw - sw));
}

template <typename Real>
__device__ __forceinline__ Real rcp_(Real x)
{
    if constexpr (std::is_same<Real, double>::value) return 1.0 / x;
    else return __frcp_rn(x);
}

// Loads of one row for the pull: populations of one lattice (plane base pointers `pl`,
// wall rule KIND) at row y and column x, with the wall rules of Sec. 5.1.  Offsets are
// 32-bit element indices; the row part is CTA-uniform.
template <int KIND, int Q, typename Real, typename Store>
__device__ __forceinline__ void pull_row_(const Store *const *pl, int pitch, int ny, int nx, int y, int x, int xm,
                                          int xp, Real iscale, const Real *__restrict__ twall, Real dTcold, Real *out)
{
    const int r0 = y * pitch;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int ex = ex_(a), ey = ey_(a);
        const int xs = ex > 0 ? xm : (ex < 0 ? xp : x);
        const bool wall = (ey > 0 && y == 0) || (ey < 0 && y == ny - 1);
        Real v;
        if (!wall) {
            const int rs = ey > 0 ? r0 - pitch : (ey < 0 ? r0 + pitch : r0);
            v = ld_<Real, Store>(pl[a] + (rs + xs));
        } else if (KIND == 0) {
            v = ld_<Real, Store>(pl[mir_(a)] + (r0 + xs));
        } else {
            v = ld_<Real, Store>(pl[opp_(a)] + (r0 + x));
        }
        if constexpr (scaled_<Store>()) v *= iscale;
        if (KIND == 2 && wall) {
            const Real tw = ey > 0 ? twall[(1 - ex) * nx + x] : dTcold;
            v = -v + Real(2.0 * w_<Q>(a)) * tw;
        }
        out[a] = v;
    }
}

template <typename Real, typename Store, int QF, int QT, int TX>
__device__ __forceinline__ void march_body(const StepArgs<Real, Store> &A, int seg, int bx, int by)
{
    using R2 = typename Vec2<Real>::T;
    constexpr int PX = TX + 4, SX = TX + 2;
    __shared__ Real s_phi[8][PX];
    __shared__ R2 s_sp[4][SX];   // (sigma - sigma0, p - p0)
    __shared__ R2 s_n[4][SX];    // unit normal

    const int nx = A.nx, ny = A.ny, pitch = A.pitch;
    const long long plane = A.plane;
    const Phys<Real> &P = A.P;
    const int tid = threadIdx.x;
    const int x0 = bx * TX;
    const int y0 = by * seg;
    const int y1 = min(y0 + seg, ny);
    const int x = x0 + tid;
    const bool xin = x < nx;
    const int xw = wrap_(x, nx);
    const int xm = xw == 0 ? nx - 1 : xw - 1, xp = xw == nx - 1 ? 0 : xw + 1;
    const int hpc = tid < 2 ? tid : TX + tid;               // phi halo tile column (tid < 4)
    const int hpx = wrap_(x0 - 2 + hpc, nx);
    const int hpxm = hpx == 0 ? nx - 1 : hpx - 1, hpxp = hpx == nx - 1 ? 0 : hpx + 1;
    const int hsc = tid == 0 ? 0 : TX + 1;                  // sigma/n halo tile column (tid < 2)
    const int hsx = wrap_(x0 - 1 + hsc, nx);
    const int hsxm = hsx == 0 ? nx - 1 : hsx - 1, hsxp = hsx == nx - 1 ? 0 : hsx + 1;

    // Row inputs: f of the thread's column (for phi and the collision) and, on threads
    // 0..3, f of one phi halo column; h and p of the thread's column and, on threads 0..1,
    // of one sigma halo column.  All of them are loaded one row ahead of their use.
    struct RowF {
        Real f[QF], fh[QF];
    };
    struct RowH {
        Real h[QT], hh[QT], dp, dph;
    };
    auto load_f = [&](int r, RowF &q) {
        const int gy = mirror_row_(r, ny);
        pull_row_<0, QF>(A.fi, pitch, ny, nx, gy, xw, xm, xp, A.isf, A.twall, P.dTcold, q.f);
        if (tid < 4) pull_row_<0, QF>(A.fi, pitch, ny, nx, gy, hpx, hpxm, hpxp, A.isf, A.twall, P.dTcold, q.fh);
    };
    auto load_h = [&](int r, RowH &q) {
        const int gy = mirror_row_(r, ny);
        pull_row_<2, QT>(A.hi, pitch, ny, nx, gy, xw, xm, xp, A.ish, A.twall, P.dTcold, q.h);
        q.dp = A.dp_in[gy * pitch + xw];
        if (tid < 2) {
            pull_row_<2, QT>(A.hi, pitch, ny, nx, gy, hsx, hsxm, hsxp, A.ish, A.twall, P.dTcold, q.hh);
            q.dph = A.dp_in[gy * pitch + hsx];
        }
    };
    auto put_phi = [&](int r, const RowF &q) {
        Real phi = q.f[0];
#pragma unroll
        for (int a = 1; a < QF; ++a) phi += q.f[a];
        s_phi[r & 7][tid + 2] = phi;
        if (tid < 4) {
            Real ph = q.fh[0];
#pragma unroll
            for (int a = 1; a < QF; ++a) ph += q.fh[a];
            s_phi[r & 7][hpc] = ph;
        }
    };
    auto sig_of = [&](int r, Real dT, int col) -> Real {
        if (r == -1) dT = Real(2) * A.twall[nx + col] - dT;   // T_ghost = 2 T_w - T_adjacent
        else if (r == ny) dT = Real(2) * P.dTcold - dT;
        return dT * (P.sigma1 + P.sigma2 * dT);
    };
    auto put_sig = [&](int r, const RowH &q) {
        Real dT = q.h[0];
#pragma unroll
        for (int a = 1; a < QT; ++a) dT += q.h[a];
        R2 v;
        v.x = sig_of(r, dT, xw);
        v.y = q.dp;
        s_sp[r & 3][tid + 1] = v;
        if (tid < 2) {
            Real d = q.hh[0];
#pragma unroll
            for (int a = 1; a < QT; ++a) d += q.hh[a];
            R2 w;
            w.x = sig_of(r, d, hsx);
            w.y = q.dph;
            s_sp[r & 3][hsc] = w;
        }
    };
    auto put_n = [&](int r) {
        const Real *rm = s_phi[(r - 1) & 7], *r0 = s_phi[r & 7], *rp = s_phi[(r + 1) & 7];
        Real gx, gy;
        R2 n;
        grad3_(rm, r0, rp, tid + 2, gx, gy);
        unit_normal_(gx, gy, P.g2min, n.x, n.y);
        s_n[r & 3][tid + 1] = n;
        if (tid < 2) {
            grad3_(rm, r0, rp, hsc + 1, gx, gy);
            unit_normal_(gx, gy, P.g2min, n.x, n.y);
            s_n[r & 3][hsc] = n;
        }
    };

    // ---- prologue: phi rows y0-2 .. y0+1, sigma/p rows y0-1, y0, normals y0-1, y0 ----
    Real fq0[QF], fq1[QF], hq0[QT], gn[9];
    RowF fn;
    RowH hn;
    {
        RowF t;
        RowH th;
        load_f(y0 - 2, t);
        put_phi(y0 - 2, t);
        load_f(y0 - 1, t);
        put_phi(y0 - 1, t);
        load_f(y0, t);
        put_phi(y0, t);
#pragma unroll
        for (int a = 0; a < QF; ++a) fq0[a] = t.f[a];
        load_f(y0 + 1, t);
        put_phi(y0 + 1, t);
#pragma unroll
        for (int a = 0; a < QF; ++a) fq1[a] = t.f[a];
        load_h(y0 - 1, th);
        put_sig(y0 - 1, th);
        load_h(y0, th);
        put_sig(y0, th);
#pragma unroll
        for (int a = 0; a < QT; ++a) hq0[a] = th.h[a];
    }
    // next row's loads: f(y0+2), h(y0+1), g(y0)
    load_f(y0 + 2, fn);
    load_h(y0 + 1, hn);
    pull_row_<1, 9>(A.gi, pitch, ny, nx, y0, xw, xm, xp, A.isg, A.twall, P.dTcold, gn);
    __syncthreads();
    put_n(y0 - 1);
    put_n(y0);

    const Real c2 = Real(1.0 / 3.0), hf = Real(0.5);
    for (int y = y0; y < y1; ++y) {
        Real fq2[QF], hq1[QT], g[9];
#pragma unroll
        for (int a = 0; a < QF; ++a) fq2[a] = fn.f[a];
#pragma unroll
        for (int a = 0; a < QT; ++a) hq1[a] = hn.h[a];
#pragma unroll
        for (int a = 0; a < 9; ++a) g[a] = gn[a];
        put_phi(y + 2, fn);
        put_sig(y + 1, hn);
        // issue the loads of the next row before this row's barriers and collisions
        if (y + 1 < y1) {
            load_f(y + 3, fn);
            load_h(y + 2, hn);
            pull_row_<1, 9>(A.gi, pitch, ny, nx, y + 1, xw, xm, xp, A.isg, A.twall, P.dTcold, gn);
        }
        __syncthreads();
        put_n(y + 1);
        __syncthreads();
        if (xin) {
            const int c = tid + 2, s = tid + 1;
            const Real *pm = s_phi[(y - 1) & 7], *p0 = s_phi[y & 7], *pp = s_phi[(y + 1) & 7];
            const Real phi = p0[c];
            Real gpx, gpy;
            grad3_(pm, p0, pp, c, gpx, gpy);
            const Real g2 = gpx * gpx + gpy * gpy;
            const R2 *nm = s_n[(y - 1) & 3], *n0 = s_n[y & 3], *np = s_n[(y + 1) & 3];
            const R2 *qm = s_sp[(y - 1) & 3], *q0 = s_sp[y & 3], *qp = s_sp[(y + 1) & 3];
            const R2 nC = n0[s], nE = n0[s + 1], nW = n0[s - 1], nN = np[s], nS = nm[s];
            const R2 nNE = np[s + 1], nNW = np[s - 1], nSE = nm[s + 1], nSW = nm[s - 1];
            const Real c1 = Real(1.0 / 3.0), cd = Real(1.0 / 12.0);
            const Real divn = c1 * (nE.x - nW.x) + cd * ((nNE.x - nNW.x) + (nSE.x - nSW.x)) + c1 * (nN.y - nS.y) +
                              cd * ((nNE.y - nSE.y) + (nNW.y - nSW.y));
            const R2 qE = q0[s + 1], qW = q0[s - 1], qN = qp[s], qS = qm[s];
            const R2 qNE = qp[s + 1], qNW = qp[s - 1], qSE = qm[s + 1], qSW = qm[s - 1];
            const Real dsx = c1 * (qE.x - qW.x) + cd * ((qNE.x - qNW.x) + (qSE.x - qSW.x));
            const Real dsy = c1 * (qN.x - qS.x) + cd * ((qNE.x - qSE.x) + (qNW.x - qSW.x));
            const Real dpx = c1 * (qE.y - qW.y) + cd * ((qNE.y - qNW.y) + (qSE.y - qSW.y));
            const Real dpy = c1 * (qN.y - qS.y) + cd * ((qNE.y - qSE.y) + (qNW.y - qSW.y));
            const Real nxv = nC.x, nyv = nC.y;
            Real dT = hq0[0];
#pragma unroll
            for (int a = 1; a < QT; ++a) dT += hq0[a];
            const Real sigma = P.sigma0 + dT * (P.sigma1 + P.sigma2 * dT);
            const Real Fsx = P.csf * (-sigma * g2 * divn * nxv + g2 * ((Real(1) - nxv * nxv) * dsx - nxv * nyv * dsy));
            const Real Fsy = P.csf * (-sigma * g2 * divn * nyv + g2 * ((Real(1) - nyv * nyv) * dsy - nxv * nyv * dsx));
            const Real Ftx = Fsx + P.Fx, Fty = Fsy + P.Fy;
            const Real Fpx = -dpx + c2 * P.drho * gpx, Fpy = -dpy + c2 * P.drho * gpy;
            const Real rho = P.rhoA + phi * P.drho;
            const Real irho = rcp_(rho);
            const Real s0 = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
            const Real sx = (g[1] - g[3]) + ((g[5] - g[6]) + (g[8] - g[7]));
            const Real sy = (g[2] - g[4]) + ((g[5] + g[6]) - (g[7] + g[8]));
            const Real irc2 = Real(3) * irho;
            const Real ux = (sx + hf * c2 * Ftx) * irc2;
            const Real uy = (sy + hf * c2 * Fty) * irc2;
            const Real dp = s0 + hf * (Fpx * ux + Fpy * uy);
            const Real om_nu = rcp_(Real(3) * (P.muA + phi * P.dmu) * irho + hf);
            const Real om_T = rcp_(Real(3) * (P.kA + phi * P.dk) * irho + hf);
            const Real theta = P.W4 * phi * (Real(1) - phi);
            collide_phase_<QF>(fq0, phi, ux, uy, P.Mphi * theta * nxv, P.Mphi * theta * nyv, P.omega_phi);
            collide_flow_(g, rho, dp, ux, uy, Fpx, Fpy, Ftx, Fty, om_nu, s0, sx, sy);
            collide_energy_<QT>(hq0, dT, ux, uy, P.T_ref, om_T);
            const int o = y * pitch + x;
#pragma unroll
            for (int a = 0; a < QF; ++a) {
                Real v = fq0[a];
                if constexpr (scaled_<Store>()) v *= A.sf;
                st_(A.fo[a] + o, v);
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                Real v = g[a];
                if constexpr (scaled_<Store>()) v *= A.sg;
                st_(A.go[a] + o, v);
            }
#pragma unroll
            for (int a = 0; a < QT; ++a) {
                Real v = hq0[a];
                if constexpr (scaled_<Store>()) v *= A.sh;
                st_(A.ho[a] + o, v);
            }
            A.dp_out[o] = dp;
            if (A.macro) {
                const long long N = (long long)nx * ny, m = (long long)y * nx + x;
                A.macro[m] = double(phi);
                A.macro[N + m] = double(ux);
                A.macro[2 * N + m] = double(uy);
                A.macro[3 * N + m] = double(P.T_ref) + double(dT);
                A.macro[4 * N + m] = double(dp);
            }
        }
#pragma unroll
        for (int a = 0; a < QF; ++a) {
            fq0[a] = fq1[a];
            fq1[a] = fq2[a];
        }
#pragma unroll
        for (int a = 0; a < QT; ++a) hq0[a] = hq1[a];
    }
}

template <typename Real, typename Store, int QF, int QT, int TX>
__global__ void __launch_bounds__(TX, 2) march_kernel(const StepArgs<Real, Store> A, int seg)
{
    march_body<Real, Store, QF, QT, TX>(A, seg, blockIdx.x, blockIdx.y);
}

// Many channels of uneven size in one launch: CTA i works on strip ctas[i].y, segment
// ctas[i].z of case ctas[i].x, with that case's arguments; cases whose active flag is 0
// (converged) are skipped.
template <typename Real, typename Store, int QF, int QT, int TX>
__global__ void __launch_bounds__(TX, 2) batch_kernel(const StepArgs<Real, Store> *__restrict__ cases,
                                                       const int4 *__restrict__ ctas, const int *__restrict__ active,
                                                       int seg)
{
    const int4 t = ctas[blockIdx.x];
    if (!active[t.x]) return;
    march_body<Real, Store, QF, QT, TX>(cases[t.x], seg, t.y, t.z);
}

template <typename Real> constexpr int march_width() { return std::is_same<Real, double>::value ? 128 : 256; }

template <typename Real, typename Store, int QF, int QT>
int step_strip_width()
{
    return march_width<Real>();
}

template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_batch(const StepArgs<Real, Store> *cases, const int4 *ctas, int n_ctas, const int *active, int seg,
                         cudaStream_t s)
{
    constexpr int TX = march_width<Real>();
    batch_kernel<Real, Store, QF, QT, TX><<<n_ctas, TX, 0, s>>>(cases, ctas, active, seg);
    return cudaGetLastError();
}

template <typename Real, typename Store, int QF, int QT>
int resident_ctas()
{
    constexpr int TX = march_width<Real>();
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<Real, Store, QF, QT, TX>, TX, 0);
    return sms * (per_sm > 0 ? per_sm : 1);
}

// Segment length: the grid (strips x segments) is made as close as possible to a whole
// number of waves of resident CTAs, preferring long segments (each segment re-derives 4
// rows of phi and 2 of sigma to start its window).
static int choose_segment(int strips, int ny, int slots)
{
    int best = ny, best_key = -1;
    for (int nseg = 1; nseg <= (ny + 7) / 8; ++nseg) {
        const int seg = (ny + nseg - 1) / nseg;
        const int used = (ny + seg - 1) / seg;          // segments actually launched
        const long long ctas = (long long)strips * used;
        const long long waves = (ctas + slots - 1) / slots;
        // efficiency in per-mille, then longer segments first
        const int eff = int(1000 * ctas / (waves * slots));
        const int warm = int(1000 * 6 / (seg + 6));     // start-up rows per segment
        const int key = eff - warm;
        if (key > best_key) {
            best_key = key;
            best = seg;
        }
    }
    return best;
}

template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_step(const StepArgs<Real, Store> &A, cudaStream_t s, int seg_rows)
{
    // FP64 needs ~240 registers per thread: 128-thread strips; otherwise 256
    constexpr int TX = march_width<Real>();
    static int slots = 0;   // resident CTAs on the device (per template instance)
    if (slots == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_kernel<Real, Store, QF, QT, TX>, TX, 0);
        slots = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int strips = (A.nx + TX - 1) / TX;
    const int seg = seg_rows > 0 ? (seg_rows < A.ny ? seg_rows : A.ny) : choose_segment(strips, A.ny, slots);
    dim3 grid(strips, (A.ny + seg - 1) / seg);
    march_kernel<Real, Store, QF, QT, TX><<<grid, TX, 0, s>>>(A, seg);
    return cudaGetLastError();
}

#define LBM_INST(R, S, QF, QT)                                                                              \
    template cudaError_t launch_step<R, S, QF, QT>(const StepArgs<R, S> &, cudaStream_t, int);             \
    template cudaError_t launch_batch<R, S, QF, QT>(const StepArgs<R, S> *, const int4 *, int, const int *, \
                                                    int, cudaStream_t);                                   \
    template int step_strip_width<R, S, QF, QT>();                                                         \
    template int resident_ctas<R, S, QF, QT>();
LBM_INST(double, double, 5, 5)
LBM_INST(double, double, 5, 9)
LBM_INST(double, double, 9, 5)
LBM_INST(double, double, 9, 9)
LBM_INST(float, float, 5, 5)
LBM_INST(float, float, 5, 9)
LBM_INST(float, float, 9, 5)
LBM_INST(float, float, 9, 9)
LBM_INST(float, __half, 5, 5)
LBM_INST(float, __half, 5, 9)
LBM_INST(float, __half, 9, 5)
LBM_INST(float, __half, 9, 9)
#undef LBM_INST

}  // namespace lbm
