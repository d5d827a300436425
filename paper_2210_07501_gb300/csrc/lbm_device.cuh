// lbm_device.cuh -- device-side building blocks of the GB300 coupled central-moment LB
// step (arXiv 2210.07501, Sec. 4.1-4.3, App. B): lattice constants, storage conversion,
// pull streaming with the wall rules of Sec. 5.1, isotropic stencils and the three
// central-moment collisions in closed form.
//
// Variables carried (exact affine changes of the paper's variables):
//   f - r(y)   phase-field populations (Sec. 4.1) minus those of a reference state r that
//              depends on the row only: the flat tanh interface of width W at y = b, at
//              rest, at its central-moment equilibrium (first moment M_phi theta, the
//              normal pointing up);
//   g - w p0   flow populations minus the rest weights times p0 = rho_A c^2 (Sec. 4.2);
//   h - w Tr   energy populations minus the rest weights times T_ref (Sec. 4.3);
//   dp = p - p0.
// The velocity is ~1e-5 of p and the interface tilt that drives it is a ~1e-5 change of
// phi ~ 1, so carrying deviations keeps round-off far below the signal: phi - phi0(y),
// its gradient, the normal's n_y - 1 and the collision's output are formed from small
// numbers and never from differences of O(1) ones.  Equilibria are the printed ones
// minus the central moments of the subtracted reference, written without cancellation.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// ---- D2Q9 velocities (Sec. 4.1; velocity 8 is (+1,-1) as in App. B's P) ----
__host__ __device__ constexpr int ex_(int a) { return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey_(int a) { return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0); }
// reversed velocity (bounce-back) and velocity mirrored in y (specular reflection)
__host__ __device__ constexpr int opp_(int a) { return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4 + 1) : ((a - 3) % 4 + 5)); }
__host__ __device__ constexpr int mir_(int a)
{
    return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}
// weights: D2Q9 (4/9, 1/9, 1/36); D2Q5 (1/3, 1/6); c^2 = 1/3 for both
template <int Q>
__host__ __device__ constexpr double w_(int a)
{
    return Q == 9 ? (a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0)) : (a == 0 ? 1.0 / 3.0 : 1.0 / 6.0);
}

template <typename Real> struct Phys {
    Real W4;          // 4 / W          (sharpening theta = W4 phi (1 - phi))
    Real csf;         // 1.5 W          (delta_s = 1.5 W |grad phi|^2)
    Real sigma0, sigma1, sigma2;
    Real T_ref;
    Real dTcold;      // T_cold - T_ref
    Real rhoA, drho;  // rho(phi) = rhoA + phi drho
    Real muA, dmu;    // mu(phi)
    Real kA, dk;      // k(phi), c_p = 1
    Real omega_phi, Mphi;
    Real Fx, Fy;
    Real g2min;       // |grad phi|^2 below which n = 0
};

template <typename Real, typename Store> struct StepArgs {
    int nx, ny, pitch;
    long long plane;                // ny * pitch elements per population plane
    const Store *f_in;
    Store *f_out;
    const Store *g_in;
    Store *g_out;
    const Store *h_in;
    Store *h_out;
    const Real *dp_in;              // p - p0 of the previous step [ny][pitch]
    Real *dp_out;
    const Real *twall;              // [3][nx]: T_w - T_ref at x - 1/2, x, x + 1/2 (bottom wall)
    // per-row tables of the phase-field reference, [RT_N][ny + 2], row r at index r + 1:
    // phi0(r) = sum_a r_a(r), dR(r) = (sum of the pulled reference populations) - phi0(r)
    // (as high and low parts in FP32), the normal's reference gradient d_y phi0 (r = -1 ..
    // ny, ghost rows mirrored), theta(phi0(r)) and the first-moment constant
    // c01(r) = (1 - omega_phi) Ry(r) + omega_phi M_phi theta(phi0(r)) - t01(r), Ry the first
    // y moment of the pulled reference populations and t01 that of r itself
    const Real *rtab;
    // the same values regrouped per output row y, [ny][RX_N]: what the row-marching kernel
    // needs at row y, staged in shared memory with the row's population copies
    const Real *rowx;
    const double *phi0;             // [ny]: phi0 in FP64 (field export)
    const double *fref;             // [QF][ny]: the reference populations r_a(y) in FP64
    double *macro;                  // optional [5][ny][nx]: phi, u, v, T, dp
    // per-population plane base pointers (plane a of lattice X starts at X_in + a * plane)
    const Store *fi[9], *gi[9], *hi[9];
    Store *fo[9], *go[9], *ho[9];
    Phys<Real> P;
    Real sf, sg, sh;                // storage scales (value * s is stored); 1 unless FP16
    Real isf, isg, ish;
    unsigned int *fault;            // set to nonzero by a CTA that abandoned the step
    unsigned int tx_extra;          // bytes each stage expects beyond its copies: 0 (test hook)
};

// rows of StepArgs::rtab
enum { RT_PHI0 = 0, RT_DR = 1, RT_GREF = 2, RT_TH0 = 3, RT_C01 = 4, RT_DRLO = 5, RT_N = 6 };
// fields of StepArgs::rowx for output row y: phi0(y), theta(phi0(y)), c01(y), d_y phi0(y),
// dR of the mirrored row y + 3 (high, low), d_y phi0(y + 1), unused
enum { RX_PHI0 = 0, RX_TH0 = 1, RX_C01 = 2, RX_GREF = 3, RX_DR3 = 4, RX_DR3LO = 5, RX_GREF1 = 6, RX_N = 8 };

// ---- storage conversion ----
template <typename Real, typename Store>
__device__ __forceinline__ Real ld_(const Store *p)
{
    if constexpr (std::is_same<Store, __half>::value)
        return Real(__half2float(__ldg(p)));
    else
        return Real(__ldg(p));
}
template <typename Real, typename Store>
__device__ __forceinline__ void st_(Store *p, Real v)
{
    if constexpr (std::is_same<Store, __half>::value)
        *p = __float2half_rn(float(v));
    else
        *p = Store(v);
}
template <typename Store> constexpr bool scaled_() { return std::is_same<Store, __half>::value; }

__device__ __forceinline__ int wrap_(int x, int n)
{
    int r = x % n;
    return r < 0 ? r + n : r;
}
// ghost rows mirror the nearest interior rows (zero normal gradient); rows further out
// than the stencils reach are clamped (they are never used by a lattice node)
__device__ __forceinline__ int mirror_row_(int y, int ny)
{
    if (y < 0) y = -1 - y;
    if (y >= ny) y = 2 * ny - 1 - y;
    return y < 0 ? 0 : (y >= ny ? ny - 1 : y);
}


// ---- isotropic finite differences on a shared-memory tile:
// d_i psi = (1/c^2) sum_a w_a e_ai psi(x + e_a) with the D2Q9 weights ----
template <typename Real, int LD>
__device__ __forceinline__ void iso_grad_(const Real (*s)[LD], int y, int x, Real &gx, Real &gy)
{
    const Real c1 = Real(1.0 / 3.0), c2 = Real(1.0 / 12.0);
    const Real ne = s[y + 1][x + 1], nw = s[y + 1][x - 1], se = s[y - 1][x + 1], sw = s[y - 1][x - 1];
    gx = c1 * (s[y][x + 1] - s[y][x - 1]) + c2 * ((ne - nw) + (se - sw));
    gy = c1 * (s[y + 1][x] - s[y - 1][x]) + c2 * ((ne - se) + (nw - sw));
}

template <typename Real>
__device__ __forceinline__ void unit_normal_(Real gx, Real gy, Real g2min, Real &nx, Real &ny)
{
    const Real g2 = gx * gx + gy * gy;
    if (g2 > g2min) {
        if constexpr (std::is_same<Real, double>::value) {
            const double m = sqrt(g2);
            nx = gx / m;
            ny = gy / m;
        } else {
            const float r = rsqrtf(g2);
            nx = gx * r;
            ny = gy * r;
        }
    } else {
        nx = Real(0);
        ny = Real(0);
    }
}

// Reciprocal: IEEE in FP64; in FP32 the hardware approximation (about 1 ulp): the
// operands are densities, relaxation rates and gradient norms of order one or above the
// normal's threshold, and FP32 storage dominates the error budget.
template <typename Real>
__device__ __forceinline__ Real rcp_(Real x)
{
    if constexpr (std::is_same<Real, double>::value) {
        return 1.0 / x;
    } else {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
}

// The unit normal n = grad phi / |grad phi| as (n_x, n_y - 1).  For an interface close to
// the flat reference n_y is close to 1, so n_y - 1 = -g_x^2 / (|g| (|g| + g_y)) is formed
// without cancellation; the stencils of div n take its differences.  n = 0 (n_y - 1 = -1)
// where |grad phi|^2 <= g2min.
template <typename Real>
__device__ __forceinline__ void unit_normal_dev_(Real gx, Real gy, Real g2min, Real &nx, Real &my)
{
    const Real g2 = gx * gx + gy * gy;
    if (g2 > g2min) {
        Real m, im;
        if constexpr (std::is_same<Real, double>::value) {
            m = sqrt(g2);
            im = 1.0 / m;
        } else {
            im = rsqrtf(g2);
            m = g2 * im;
        }
        nx = gx * im;
        my = gy > Real(0) ? -gx * nx * rcp_(m + gy) : gy * im - Real(1);
    } else {
        nx = Real(0);
        my = Real(-1);
    }
}

// ---- FP32 forms with the x and y halves paired: one packed instruction (sm_100 and
// later) does both halves of an operation.  Same terms as the generic forms below, partly
// summed in another order; used for FP32 arithmetic only (FP64 keeps the generic forms). ----
__device__ __forceinline__ float2 f2_(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc2_(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2_(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2_(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2_(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// D2Q9 central moments -> populations (see central_to_pop9_), FP32.  SCALED: the results
// come out multiplied by the storage scale so (FP16 storage), folded into the constants.
template <bool REST_LAST, bool SCALED = false>
__device__ __forceinline__ void central_to_pop9_f_(const float dk[9], const float k[9], float ux, float uy, float g[9],
                                                   float so = 1.f)
{
    const float hs = SCALED ? 0.5f * so : 0.5f, qs = SCALED ? 0.25f * so : 0.25f;
    const float2 U = f2_(ux, uy), U2 = mul2_(U, U);
    const float ux2 = U2.x, uy2 = U2.y, uxy = ux * uy;
    const float r00 = dk[0];
    const float2 R1 = fma2_(U, bc2_(k[0]), f2_(dk[1], dk[2]));                                         // r10, r01
    const float2 R2 = fma2_(U2, bc2_(k[0]), fma2_(add2_(U, U), f2_(k[1], k[2]), f2_(dk[3], dk[4])));   // r20, r02
    const float r11 = dk[5] + uy * k[1] + ux * k[2] + uxy * k[0];
    const float r21 = dk[6] + 2.f * ux * k[5] + uy * k[3] + ux2 * k[2] + 2.f * uxy * k[1] + ux2 * uy * k[0];
    const float r12 = dk[7] + 2.f * uy * k[5] + ux * k[4] + uy2 * k[1] + 2.f * uxy * k[2] + ux * uy2 * k[0];
    const float r22 = dk[8] + 2.f * ux * k[7] + 2.f * uy * k[6] + ux2 * k[4] + uy2 * k[3] + 4.f * uxy * k[5] +
                      2.f * uxy * uy * k[1] + 2.f * uxy * ux * k[2] + ux2 * uy2 * k[0];
    const float2 Q = f2_(r12, r21), W = f2_(r11, r22);
    const float2 E = sub2_(R2, bc2_(r22));   // r20 - r22, r02 - r22
    const float2 V = sub2_(R1, Q);            // r10 - r12, r01 - r21
    const float2 G12 = mul2_(bc2_(hs), add2_(E, V));   // g1, g2
    const float2 G34 = mul2_(bc2_(hs), sub2_(E, V));   // g3, g4
    const float2 S = add2_(W, Q);                         // r11 + r12, r22 + r21
    const float2 D = sub2_(W, Q);                         // r11 - r12, r22 - r21
    g[1] = G12.x;
    g[2] = G12.y;
    g[3] = G34.x;
    g[4] = G34.y;
    g[5] = qs * (S.x + S.y);
    g[6] = qs * (S.y - S.x);
    g[7] = qs * (D.x + D.y);
    g[8] = qs * (D.y - D.x);
    if constexpr (REST_LAST) {
        const float2 P = add2_(G12, G34);
        const float rest = (P.x + P.y) + ((g[5] + g[6]) + (g[7] + g[8]));
        g[0] = SCALED ? r00 * so - rest : r00 - rest;
    } else {
        g[0] = r00 - R2.x - R2.y + r22;
        if constexpr (SCALED) g[0] *= so;
    }
}

// D2Q5 central moments -> populations (see central_to_pop5_), FP32: dk = (dk0, DK1, DK2),
// k = (k0, K1, .) as pairs (first and second moments), U = (ux, uy), U2 = (ux^2, uy^2);
// SCALED as for central_to_pop9_f_
template <bool REST_LAST, bool SCALED = false>
__device__ __forceinline__ void central_to_pop5_f_(float dk0, float2 DK1, float2 DK2, float k0, float2 K1, float2 U,
                                                   float2 U2, float f[5], float so = 1.f)
{
    const float hs = SCALED ? 0.5f * so : 0.5f;
    const float2 R1 = fma2_(U, bc2_(k0), DK1);                            // r10, r01
    const float2 R2 = fma2_(U2, bc2_(k0), fma2_(add2_(U, U), K1, DK2));   // r20, r02
    const float2 A = mul2_(bc2_(hs), add2_(R1, R2));                      // f1, f2
    const float2 B = mul2_(bc2_(hs), sub2_(R2, R1));                      // f3, f4
    f[1] = A.x;
    f[2] = A.y;
    f[3] = B.x;
    f[4] = B.y;
    if constexpr (REST_LAST) {
        const float2 S = add2_(A, B);
        f[0] = SCALED ? dk0 * so - (S.x + S.y) : dk0 - (S.x + S.y);
    } else {
        f[0] = dk0 - R2.x - R2.y;
        if constexpr (SCALED) f[0] *= so;
    }
}

// ---- App. B: central moments -> populations, F(-u) then P^-1 (D2Q9).
// Moment order 00, 10, 01, 20, 02, 11, 21, 12, 22. ----
// dk: the central moments minus those of a reference at u = 0 (whose raw moments they
// are), k: the full central moments.  Raw moments r = F(-u) k = k + (F(-u) - I) k, so the
// deviation of r from the reference is dk + (F(-u) - I) k: every term of the second part
// carries a velocity factor.  With dk = k this is the plain map.
// REST_LAST: the rest population is formed last as r00 - (sum of the others), so that the
// populations sum to the conserved zeroth moment up to one rounding of a small number
// (measured on a float32 conduction lattice: the T error after 2000 steps falls from
// 2.9e-6 to 1.8e-7, the level of float32 storage alone); used for the conserved scalar
// lattices (phi, T).
// SCALED (FP32 arithmetic only): results multiplied by the storage scale so.
template <typename Real, bool REST_LAST = false, bool SCALED = false>
__device__ __forceinline__ void central_to_pop9_(const Real dk[9], const Real k[9], Real ux, Real uy, Real g[9],
                                                 Real so = Real(1))
{
    static_assert(!SCALED || std::is_same<Real, float>::value, "storage scales go with FP32 arithmetic");
    if constexpr (std::is_same<Real, float>::value) {
        central_to_pop9_f_<REST_LAST, SCALED>(dk, k, ux, uy, g, so);
        return;
    }
    const Real ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const Real r00 = dk[0];
    const Real r10 = dk[1] + ux * k[0];
    const Real r01 = dk[2] + uy * k[0];
    const Real r20 = dk[3] + Real(2) * ux * k[1] + ux2 * k[0];
    const Real r02 = dk[4] + Real(2) * uy * k[2] + uy2 * k[0];
    const Real r11 = dk[5] + uy * k[1] + ux * k[2] + uxy * k[0];
    const Real r21 = dk[6] + Real(2) * ux * k[5] + uy * k[3] + ux2 * k[2] + Real(2) * uxy * k[1] + ux2 * uy * k[0];
    const Real r12 = dk[7] + Real(2) * uy * k[5] + ux * k[4] + uy2 * k[1] + Real(2) * uxy * k[2] + ux * uy2 * k[0];
    const Real r22 = dk[8] + Real(2) * ux * k[7] + Real(2) * uy * k[6] + ux2 * k[4] + uy2 * k[3] +
                     Real(4) * uxy * k[5] + Real(2) * uxy * uy * k[1] + Real(2) * uxy * ux * k[2] + ux2 * uy2 * k[0];
    const Real h = Real(0.5), q = Real(0.25);
    g[1] = h * (r10 + r20 - r12 - r22);
    g[2] = h * (r01 + r02 - r21 - r22);
    g[3] = h * (-r10 + r20 + r12 - r22);
    g[4] = h * (-r01 + r02 + r21 - r22);
    g[5] = q * (r11 + r21 + r12 + r22);
    g[6] = q * (-r11 + r21 - r12 + r22);
    g[7] = q * (r11 - r21 - r12 + r22);
    g[8] = q * (-r11 - r21 + r12 + r22);
    if constexpr (REST_LAST)
        g[0] = r00 - (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
    else
        g[0] = r00 - r20 - r02 + r22;
}

// D2Q5 analogue: basis 1, e_x, e_y, e_x^2, e_y^2 (the first five rows of F(-u)).
template <typename Real, bool REST_LAST = false, bool SCALED = false>
__device__ __forceinline__ void central_to_pop5_(const Real dk[5], const Real k[5], Real ux, Real uy, Real f[5],
                                                 Real so = Real(1))
{
    static_assert(!SCALED || std::is_same<Real, float>::value, "storage scales go with FP32 arithmetic");
    if constexpr (std::is_same<Real, float>::value) {
        const float2 U = f2_(ux, uy);
        central_to_pop5_f_<REST_LAST, SCALED>(dk[0], f2_(dk[1], dk[2]), f2_(dk[3], dk[4]), k[0], f2_(k[1], k[2]), U,
                                              mul2_(U, U), f, so);
        return;
    }
    const Real r00 = dk[0];
    const Real r10 = dk[1] + ux * k[0];
    const Real r01 = dk[2] + uy * k[0];
    const Real r20 = dk[3] + Real(2) * ux * k[1] + ux * ux * k[0];
    const Real r02 = dk[4] + Real(2) * uy * k[2] + uy * uy * k[0];
    const Real h = Real(0.5);
    f[1] = h * (r10 + r20);
    f[2] = h * (r01 + r02);
    f[3] = h * (r20 - r10);
    f[4] = h * (r02 - r01);
    f[0] = REST_LAST ? r00 - ((f[1] + f[3]) + (f[2] + f[4])) : r00 - r20 - r02;
}

template <int Q, typename Real>
__device__ __forceinline__ void raw_first_(const Real *p, Real &m10, Real &m01)
{
    if constexpr (Q == 9) {
        m10 = (p[1] - p[3]) + ((p[5] - p[6]) + (p[8] - p[7]));
        m01 = (p[2] - p[4]) + ((p[5] + p[6]) - (p[7] + p[8]));
    } else {
        m10 = p[1] - p[3];
        m01 = p[2] - p[4];
    }
}

// ---- Sec. 4.1 phase-field collision in deviation variables.  The first central moments
// relax at omega_phi towards M_phi theta n, the rest take their equilibria (phi, c^2 phi,
// c^2 phi, 0, 0, 0, c^4 phi), so of the pre-collision populations only phi and the first
// raw moments enter.  In: (m10, m01) = raw_first_ of the pulled f - r (r the reference
// populations at the rows they were pulled from), dphi = phi - phi0(y), phi, u, the normal
// (n_x, n_y - 1), theta0 = theta(phi0(y)) and dth = theta(phi) - theta0, c01 (see
// StepArgs::rtab).  Out: s = post-collision f - r(y).  With Rx = sum e_x r(pulled) = 0 (the
// reference is even in x) the pre-collision first central moments are k10 = m10 - u_x phi
// and k01 = m01 + Ry(y) - u_y phi; the reference's own post-collision first moments are
// (0, t01(y)), t01 ~ M_phi theta0. ----
// (SCALED: s comes out multiplied by the storage scale so.)
template <int Q, typename Real, bool SCALED = false>
__device__ __forceinline__ void collide_phase_dev_(Real *s, Real m10, Real m01, Real dphi, Real phi, Real ux, Real uy,
                                                   Real nx, Real my, Real th0, Real dth, Real c01, Real M, Real om,
                                                   Real so = Real(1))
{
    if constexpr (std::is_same<Real, float>::value && Q == 5) {
        const float w1 = 1.f - om, oM = om * M, c2 = 1.f / 3.f;
        const float2 U = f2_(ux, uy), NU = mul2_(bc2_(-1.f), U);
        // (t10, t01 - M theta0), then (t10, t01)
        const float2 T = fma2_(bc2_(w1), fma2_(NU, bc2_(phi), f2_(m10, m01)),
                               f2_(oM * (th0 + dth) * nx, oM * (th0 * my + dth * (1.f + my)) + c01));
        const float2 T1 = add2_(T, f2_(0.f, M * th0));
        central_to_pop5_f_<true, SCALED>(dphi, T, bc2_(c2 * dphi), phi, T1, U, mul2_(U, U), s, so);
        return;
    }
    const Real w1 = Real(1) - om, oM = om * M;
    const Real t10 = w1 * (m10 - ux * phi) + oM * (th0 + dth) * nx;
    const Real dt01 = w1 * (m01 - uy * phi) + oM * (th0 * my + dth * (Real(1) + my)) + c01;
    const Real t01 = M * th0 + dt01;
    const Real c2 = Real(1.0 / 3.0), c2d = c2 * dphi, c2p = c2 * phi;
    if constexpr (Q == 9) {
        const Real dk[9] = {dphi, t10, dt01, c2d, c2d, Real(0), Real(0), Real(0), dphi * Real(1.0 / 9.0)};
        const Real k[9] = {phi, t10, t01, c2p, c2p, Real(0), Real(0), Real(0), phi * Real(1.0 / 9.0)};
        central_to_pop9_<Real, true, SCALED>(dk, k, ux, uy, s, so);
    } else {
        const Real dk[5] = {dphi, t10, dt01, c2d, c2d};
        const Real k[5] = {phi, t10, t01, c2p, c2p};
        central_to_pop5_<Real, true, SCALED>(dk, k, ux, uy, s, so);
    }
}

// ---- Sec. 4.3 energy collision on h - w T_ref: first central moments relax at omega_T;
// the rest take (T E - T_ref Wc(u)) = dT E + T_ref D(u), where E = (1,0,0,c^2,c^2,0,0,0,c^4)
// are the Maxwellian central moments per unit T and Wc(u) those of the weights.  In: the
// pulled populations' dT = T - T_ref and first raw moments (m10, m01); out: h = the
// post-collision populations. ----
template <int Q, typename Real, bool SCALED = false>
__device__ __forceinline__ void collide_energy_(Real *h, Real m10, Real m01, Real dT, Real ux, Real uy, Real Tr, Real om,
                                                Real so = Real(1))
{
    if constexpr (std::is_same<Real, float>::value && Q == 5) {
        const float c2 = 1.f / 3.f;
        const float2 U = f2_(ux, uy), U2 = mul2_(U, U);
        const float2 K = fma2_(mul2_(bc2_(-1.f), U), bc2_(dT), f2_(m10, m01));          // k10, k01
        const float2 T = fma2_(bc2_(om), sub2_(mul2_(bc2_(Tr), U), K), K);               // t10, t01
        const float2 K2 = fma2_(bc2_(-Tr), U2, bc2_(c2 * dT));                           // k20, k02
        central_to_pop5_f_<true, SCALED>(dT, T, K2, dT, T, U, U2, h, so);
        return;
    }
    const Real k10 = m10 - ux * dT, k01 = m01 - uy * dT;
    const Real t10 = k10 + om * (Tr * ux - k10), t01 = k01 + om * (Tr * uy - k01);
    const Real c2 = Real(1.0 / 3.0);
    const Real ux2 = ux * ux, uy2 = uy * uy;
    if constexpr (Q == 9) {
        const Real k[9] = {dT,
                           t10,
                           t01,
                           c2 * dT - Tr * ux2,
                           c2 * dT - Tr * uy2,
                           -Tr * ux * uy,
                           Tr * (c2 + ux2) * uy,
                           Tr * (c2 + uy2) * ux,
                           Real(1.0 / 9.0) * dT - Tr * (c2 * (ux2 + uy2) + ux2 * uy2)};
        central_to_pop9_<Real, true, SCALED>(k, k, ux, uy, h, so);
    } else {
        const Real k[5] = {dT, t10, t01, c2 * dT - Tr * ux2, c2 * dT - Tr * uy2};
        central_to_pop5_<Real, true, SCALED>(k, k, ux, uy, h, so);
    }
}

// ---- Raw moments of the pulled flow populations that the flow step needs: the zeroth and
// first (s0, sx, sy, which give p and u, Sec. 4.2) and the second (r20, r02, r11, the F(u)
// rows of the pre-collision central moments 20, 02, 11).  FP32: from the packed sums and
// differences of (g1, g2) and (g3, g4), (g5, g7) and (g6, g8). ----
template <typename Real>
__device__ __forceinline__ void flow_raw_moments_(const Real *g, Real &s0, Real &sx, Real &sy, Real &r20, Real &r02,
                                                  Real &r11)
{
    if constexpr (std::is_same<Real, float>::value) {
        const float2 G12 = f2_(g[1], g[2]), G34 = f2_(g[3], g[4]), G57 = f2_(g[5], g[7]), G68 = f2_(g[6], g[8]);
        const float2 A = add2_(G12, G34), B = sub2_(G12, G34);   // g1 +- g3, g2 +- g4
        const float2 C = add2_(G57, G68), E = sub2_(G57, G68);   // g5 +- g6, g7 +- g8
        const float t = C.x + C.y;
        s0 = (g[0] + (A.x + A.y)) + t;
        sx = B.x + (E.x - E.y);
        sy = B.y + (C.x - C.y);
        r20 = A.x + t;
        r02 = A.y + t;
        r11 = E.x + E.y;
    } else {
        s0 = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
        sx = (g[1] - g[3]) + ((g[5] - g[6]) + (g[8] - g[7]));
        sy = (g[2] - g[4]) + ((g[5] + g[6]) - (g[7] + g[8]));
        r20 = (g[1] + g[3]) + ((g[5] + g[6]) + (g[7] + g[8]));
        r02 = (g[2] + g[4]) + ((g[5] + g[6]) + (g[7] + g[8]));
        r11 = (g[5] - g[6]) + (g[7] - g[8]);
    }
}

// ---- Sec. 4.2 two-fluid collision on g - w p0.  Only the trace-free second moment 2d
// and 11 relax at omega_nu (pre-collision values needed); every other central moment
// is replaced by equilibrium + source / 2.  Deviation equilibrium:
//   eta^eq - p0 Wc(u) = dp Wc(u) + rho c^2 D(u).  In: the pulled populations' raw moments
// (flow_raw_moments_); out: g = the post-collision populations (SCALED: multiplied by the
// storage scale so). ----
template <typename Real, bool SCALED = false>
__device__ __forceinline__ void collide_flow_(Real *g, Real rho, Real dp, Real ux, Real uy, Real Fpx, Real Fpy,
                                              Real Ftx, Real Fty, Real om, Real s0, Real sx, Real sy, Real r20,
                                              Real r02, Real r11, Real so = Real(1))
{
    static_assert(!SCALED || std::is_same<Real, float>::value, "storage scales go with FP32 arithmetic");
    if constexpr (std::is_same<Real, float>::value) {
        const float c2 = 1.f / 3.f, hf = 0.5f;
        const float2 U = f2_(ux, uy), U2 = mul2_(U, U), NU = mul2_(bc2_(-1.f), U);
        const float uxy = ux * uy;
        const float2 R2 = f2_(r20, r02);
        const float2 E = fma2_(U2, bc2_(s0), fma2_(add2_(NU, NU), f2_(sx, sy), R2));          // e20, e02
        const float e11 = r11 - uy * sx - ux * sy + uxy * s0;
        const float2 A = add2_(bc2_(c2), U2);                                                  // ax, ay
        const float rc2 = rho * c2, d = rc2 - dp;
        const float2 Q1 = mul2_(U, bc2_(d));                                                   // q10, q01
        const float2 Q2 = fma2_(bc2_(dp), A, mul2_(bc2_(-rc2), U2));                           // q20, q02
        const float q11 = -uxy * d;
        const float q21 = A.x * uy * d, q12 = A.y * ux * d;
        const float q22 = dp * A.x * A.y - rc2 * (c2 * (U2.x + U2.y) + U2.x * U2.y);
        const float G = Fpx * ux + Fpy * uy;
        const float2 S1 = fma2_(NU, bc2_(G), mul2_(bc2_(c2), f2_(Ftx, Fty)));                  // s10, s01
        const float2 S2 = fma2_(A, bc2_(G), mul2_(bc2_(2.f * c2), mul2_(f2_(Fpx, Fpy), U)));  // s20, s02
        const float s11 = c2 * (Fpx * uy + Fpy * ux) + uxy * G;
        const float sw = 1.f - hf * om;
        const float t2s = (Q2.x + Q2.y) + hf * (S2.x + S2.y);
        const float e2d = E.x - E.y;
        const float t2d = e2d + om * ((Q2.x - Q2.y) - e2d) + sw * (S2.x - S2.y);
        const float2 K1 = fma2_(bc2_(hf), S1, Q1);                                             // k10, k01
        float k[9];
        k[0] = dp + hf * G;
        k[1] = K1.x;
        k[2] = K1.y;
        k[3] = hf * (t2s + t2d);
        k[4] = hf * (t2s - t2d);
        k[5] = e11 + om * (q11 - e11) + sw * s11;
        k[6] = q21;
        k[7] = q12;
        k[8] = q22;
        central_to_pop9_f_<false, SCALED>(k, k, ux, uy, g, so);
        return;
    }
    const Real c2 = Real(1.0 / 3.0), hf = Real(0.5);
    const Real ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    // pre-collision central moments 20, 02, 11 (F(u) rows on the raw moments)
    const Real e20 = r20 - Real(2) * ux * sx + ux2 * s0;
    const Real e02 = r02 - Real(2) * uy * sy + uy2 * s0;
    const Real e11 = r11 - uy * sx - ux * sy + uxy * s0;
    // deviation equilibrium
    const Real ax = c2 + ux2, ay = c2 + uy2, rc2 = rho * c2, d = rc2 - dp;
    const Real q00 = dp, q10 = ux * d, q01 = uy * d;
    const Real q20 = dp * ax - rc2 * ux2, q02 = dp * ay - rc2 * uy2;
    const Real q11 = -uxy * d;
    const Real q21 = ax * uy * d, q12 = ay * ux * d;
    const Real q22 = dp * ax * ay - rc2 * (c2 * (ux2 + uy2) + ux2 * uy2);
    // source central moments, Gamma = F_p . u
    const Real G = Fpx * ux + Fpy * uy;
    const Real s00 = G, s10 = c2 * Ftx - ux * G, s01 = c2 * Fty - uy * G;
    const Real s20 = Real(2) * c2 * Fpx * ux + ax * G, s02 = Real(2) * c2 * Fpy * uy + ay * G;
    const Real s11 = c2 * (Fpx * uy + Fpy * ux) + uxy * G;
    // relaxation (2s at 1, 2d and 11 at omega_nu, all others at 1)
    const Real sw = Real(1) - hf * om;
    const Real t2s = (q20 + q02) + hf * (s20 + s02);
    const Real e2d = e20 - e02;
    const Real t2d = e2d + om * ((q20 - q02) - e2d) + sw * (s20 - s02);
    Real k[9];
    k[0] = q00 + hf * s00;
    k[1] = q10 + hf * s10;
    k[2] = q01 + hf * s01;
    k[3] = hf * (t2s + t2d);
    k[4] = hf * (t2s - t2d);
    k[5] = e11 + om * (q11 - e11) + sw * s11;
    k[6] = q21;
    k[7] = q12;
    k[8] = q22;
    central_to_pop9_(k, k, ux, uy, g);
}

}  // namespace lbm
