// lbm_step.cu -- the fused time step of the coupled three-lattice central-moment LB
// method (arXiv 2210.07501, Sec. 4.1-4.3) for sm_103a.
//
// One CTA owns a TX x TY tile of nodes.  Per step and node it
//   1. pulls f and h (Sec. 4.1, 4.3 streaming with the Sec. 5.1 wall rules) into
//      registers and forms phi = sum f and T - T_ref = sum h;
//   2. stages phi on a radius-2 halo, sigma(T) - sigma0 and p^{n-1} - p0 on a radius-1
//      halo in shared memory (ghost rows: phi, p mirrored; T = 2 T_w - T_adjacent);
//   3. forms the unit normal n = grad phi / |grad phi| on the radius-1 halo;
//   4. per node: curvature term div n, grad sigma, grad p, the CSF force with
//      delta_s = 1.5 W |grad phi|^2 (Sec. 3), the pressure force F_p = -grad(p - rho c^2)
//      with the stored p of the previous step, pulls g, forms u and p (Sec. 4.2), and
//      collides all three lattices in central-moment space;
//   5. writes the post-collision populations and p to the other buffer.
// Populations live in SoA planes [Q][ny][pitch], x fastest, so every pull of a warp is a
// contiguous (shifted) row segment.  No tensor cores: the step is a bandwidth-bound
// stencil.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

template <typename Real, typename Store, int QF, int QT, int BX, int BY, int RY>
__global__ void __launch_bounds__(BX *BY) step_kernel(const StepArgs<Real, Store> A)
{
    constexpr int TX = BX, TY = BY * RY;
    constexpr int PX = TX + 4, PY = TY + 4;  // phi tile with radius-2 halo
    constexpr int SX = TX + 2, SY = TY + 2;  // radius-1 tiles
    constexpr int NT = BX * BY;
    __shared__ Real s_phi[PY][PX];
    __shared__ Real s_sig[SY][SX];
    __shared__ Real s_dp[SY][SX];
    __shared__ Real s_nx[SY][SX];
    __shared__ Real s_ny[SY][SX];

    const int nx = A.nx, ny = A.ny, pitch = A.pitch;
    const long long plane = A.plane;
    const Phys<Real> &P = A.P;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    const int xg = x0 + tx;
    const int xw = wrap_(xg, nx);
    const int xm = xw == 0 ? nx - 1 : xw - 1, xp = xw == nx - 1 ? 0 : xw + 1;

    // ---- 1. own nodes: pull f and h, phi, sigma, p into the tile centre ----
    Real f[RY][QF], h[RY][QT];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int ly = ty + r * BY;
        const int yr = y0 + ly;
        const int yw = mirror_row_(yr, ny);
        pull_<0, QF>(A.f_in, plane, pitch, nx, ny, xw, xm, xp, yw, A.isf, A.twall, P.dTcold, f[r]);
        pull_<2, QT>(A.h_in, plane, pitch, nx, ny, xw, xm, xp, yw, A.ish, A.twall, P.dTcold, h[r]);
        Real phi = f[r][0], dT = h[r][0];
#pragma unroll
        for (int a = 1; a < QF; ++a) phi += f[r][a];
#pragma unroll
        for (int a = 1; a < QT; ++a) dT += h[r][a];
        if (yr == ny) dT = Real(2) * P.dTcold - dT;  // top ghost row of a ragged tile
        s_phi[ly + 2][tx + 2] = phi;
        s_sig[ly + 1][tx + 1] = dT * (P.sigma1 + P.sigma2 * dT);
        s_dp[ly + 1][tx + 1] = A.dp_in[(long long)yw * pitch + xw];
    }

    // ---- 2. halo rings ----
    for (int e = tid; e < PX * PY; e += NT) {
        const int ly = e / PX, lx = e - ly * PX;
        if (ly >= 2 && ly < TY + 2 && lx >= 2 && lx < TX + 2) continue;
        const int gx = wrap_(x0 - 2 + lx, nx);
        const int gy = mirror_row_(y0 - 2 + ly, ny);
        const int gxm = gx == 0 ? nx - 1 : gx - 1, gxp = gx == nx - 1 ? 0 : gx + 1;
        Real fr[QF];
        pull_<0, QF>(A.f_in, plane, pitch, nx, ny, gx, gxm, gxp, gy, A.isf, A.twall, P.dTcold, fr);
        Real phi = fr[0];
#pragma unroll
        for (int a = 1; a < QF; ++a) phi += fr[a];
        s_phi[ly][lx] = phi;
    }
    for (int e = tid; e < SX * SY; e += NT) {
        const int ly = e / SX, lx = e - ly * SX;
        if (ly >= 1 && ly < TY + 1 && lx >= 1 && lx < TX + 1) continue;
        const int gx = wrap_(x0 - 1 + lx, nx);
        const int yr = y0 - 1 + ly;
        const int gy = mirror_row_(yr, ny);
        const int gxm = gx == 0 ? nx - 1 : gx - 1, gxp = gx == nx - 1 ? 0 : gx + 1;
        Real hr[QT];
        pull_<2, QT>(A.h_in, plane, pitch, nx, ny, gx, gxm, gxp, gy, A.ish, A.twall, P.dTcold, hr);
        Real dT = hr[0];
#pragma unroll
        for (int a = 1; a < QT; ++a) dT += hr[a];
        if (yr == -1) dT = Real(2) * A.twall[nx + gx] - dT;   // T_ghost = 2 T_w - T_adjacent
        else if (yr == ny) dT = Real(2) * P.dTcold - dT;
        s_sig[ly][lx] = dT * (P.sigma1 + P.sigma2 * dT);
        s_dp[ly][lx] = A.dp_in[(long long)gy * pitch + gx];
    }
    __syncthreads();

    // ---- 3. unit normals on the radius-1 tile ----
    for (int e = tid; e < SX * SY; e += NT) {
        const int ly = e / SX, lx = e - ly * SX;
        Real gx, gy, nxv, nyv;
        iso_grad_<Real, PX>(s_phi, ly + 1, lx + 1, gx, gy);
        unit_normal_(gx, gy, P.g2min, nxv, nyv);
        s_nx[ly][lx] = nxv;
        s_ny[ly][lx] = nyv;
    }
    __syncthreads();

    // ---- 4./5. forces, macros, collisions, store ----
    const Real c2 = Real(1.0 / 3.0), hf = Real(0.5);
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int ly = ty + r * BY;
        const int y = y0 + ly;
        if (xg >= nx || y >= ny) continue;
        const int x = xg;
        const int cy = ly + 2, cx = tx + 2, sy1 = ly + 1, sx1 = tx + 1;
        const Real phi = s_phi[cy][cx];
        Real gpx, gpy;
        iso_grad_<Real, PX>(s_phi, cy, cx, gpx, gpy);
        const Real g2 = gpx * gpx + gpy * gpy;
        const Real nxv = s_nx[sy1][sx1], nyv = s_ny[sy1][sx1];
        const Real divn = iso_div_<Real, SX>(s_nx, s_ny, sy1, sx1);
        Real dsx, dsy, dpx, dpy;
        iso_grad_<Real, SX>(s_sig, sy1, sx1, dsx, dsy);
        iso_grad_<Real, SX>(s_dp, sy1, sx1, dpx, dpy);
        Real dT = h[r][0];
#pragma unroll
        for (int a = 1; a < QT; ++a) dT += h[r][a];
        const Real sigma = P.sigma0 + dT * (P.sigma1 + P.sigma2 * dT);
        // CSF force (Sec. 3), read with kappa = -div n and delta_s = 1.5 W |grad phi|^2
        const Real Fsx = P.csf * (-sigma * g2 * divn * nxv + g2 * ((Real(1) - nxv * nxv) * dsx - nxv * nyv * dsy));
        const Real Fsy = P.csf * (-sigma * g2 * divn * nyv + g2 * ((Real(1) - nyv * nyv) * dsy - nxv * nyv * dsx));
        const Real Ftx = Fsx + P.Fx, Fty = Fsy + P.Fy;
        // pressure force of the incompressible transformation, with the stored p^{n-1}
        const Real Fpx = -dpx + c2 * P.drho * gpx, Fpy = -dpy + c2 * P.drho * gpy;
        const Real rho = P.rhoA + phi * P.drho;

        Real g[9];
        pull_<1, 9>(A.g_in, plane, pitch, nx, ny, x, xm, xp, y, A.isg, A.twall, P.dTcold, g);
        const Real s0 = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
        const Real sx = (g[1] - g[3]) + ((g[5] - g[6]) + (g[8] - g[7]));
        const Real sy = (g[2] - g[4]) + ((g[5] + g[6]) - (g[7] + g[8]));
        const Real irc2 = Real(3) / rho;
        const Real ux = (sx + hf * c2 * Ftx) * irc2;
        const Real uy = (sy + hf * c2 * Fty) * irc2;
        const Real dp = s0 + hf * (Fpx * ux + Fpy * uy);

        // relaxation rates from the local properties (Sec. 4.1-4.3)
        const Real nu = (P.muA + phi * P.dmu) / rho;
        const Real om_nu = Real(1) / (Real(3) * nu + hf);
        const Real alpha = (P.kA + phi * P.dk) / rho;
        const Real om_T = Real(1) / (Real(3) * alpha + hf);
        const Real theta = P.W4 * phi * (Real(1) - phi);

        collide_phase_<QF>(f[r], phi, ux, uy, P.Mphi * theta * nxv, P.Mphi * theta * nyv, P.omega_phi);
        collide_flow_(g, rho, dp, ux, uy, Fpx, Fpy, Ftx, Fty, om_nu, s0, sx, sy);
        collide_energy_<QT>(h[r], dT, ux, uy, P.T_ref, om_T);

        const long long o = (long long)y * pitch + x;
#pragma unroll
        for (int a = 0; a < QF; ++a) {
            Real v = f[r][a];
            if constexpr (scaled_<Store>()) v *= A.sf;
            st_(A.f_out + a * plane + o, v);
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            Real v = g[a];
            if constexpr (scaled_<Store>()) v *= A.sg;
            st_(A.g_out + a * plane + o, v);
        }
#pragma unroll
        for (int a = 0; a < QT; ++a) {
            Real v = h[r][a];
            if constexpr (scaled_<Store>()) v *= A.sh;
            st_(A.h_out + a * plane + o, v);
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
}

template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_step(const StepArgs<Real, Store> &A, cudaStream_t s)
{
    constexpr int BX = 32, BY = 8, RY = 2;
    dim3 block(BX, BY);
    dim3 grid((A.nx + BX - 1) / BX, (A.ny + BY * RY - 1) / (BY * RY));
    step_kernel<Real, Store, QF, QT, BX, BY, RY><<<grid, block, 0, s>>>(A);
    return cudaGetLastError();
}

#define LBM_INST(R, S, QF, QT) template cudaError_t launch_step<R, S, QF, QT>(const StepArgs<R, S> &, cudaStream_t);
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
