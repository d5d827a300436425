// lbm_step.cu -- the fused time step of the coupled three-lattice central-moment LB
// method (arXiv 2210.07501, Sec. 4.1-4.3) for sm_103a.
//
// Per step and node: pull f and h (Sec. 4.1, 4.3 streaming with the Sec. 5.1 wall rules)
// and form phi = sum f and T - T_ref = sum h (phi as its deviation from the row's
// reference profile phi0, see lbm_device.cuh); stage phi (radius 2), sigma(T) - sigma0 and
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
// memory holds rings of the last rows: phi - phi0 (8 rows, radius-2 halo columns), the
// pair (sigma - sigma0, p - p0) and the unit normal as (n_x, n_y - 1) (4 rows, radius-1
// halo columns).  For output
// row y the CTA adds phi of row y + 3 (from f pulled there, whose first raw moments stay
// in registers until row y collides: the collision needs no more of them), sigma and p of
// row y + 1 (from h pulled there; T and the first raw moments kept one row), the normals of
// row y + 1, and then collides row y.  The population rows come from a ring of D stages
// in shared memory filled by bulk copies D - 1 rows ahead (below); the first rows of a
// segment are loaded directly.  Every thread works on the same row, so wall tests and row
// addresses are uniform across the CTA; only 4 halo columns per strip are recomputed.
template <typename Real> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// The RX_N reference values of a staged row (16-byte aligned) in registers: two or four
// 16-byte loads instead of one load per value.
template <typename Real>
__device__ __forceinline__ void load_rowref_(const Real *rx, Real *v)
{
    if constexpr (std::is_same<Real, float>::value) {
        const float4 a = reinterpret_cast<const float4 *>(rx)[0], b = reinterpret_cast<const float4 *>(rx)[1];
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    } else {
#pragma unroll
        for (int i = 0; i < RX_N / 2; ++i) {
            const double2 d = reinterpret_cast<const double2 *>(rx)[i];
            v[2 * i] = d.x, v[2 * i + 1] = d.y;
        }
    }
}
static_assert(RX_N == 8, "load_rowref_ reads eight values");

template <typename Real>
__device__ __forceinline__ void grad3_(const Real *rm, const Real *r0, const Real *rp, int c, Real &gx, Real &gy)
{
    const Real c1 = Real(1.0 / 3.0), c2 = Real(1.0 / 12.0);
    if constexpr (std::is_same<Real, float>::value) {
        // diagonal terms from (NE, NW) +- (SE, SW): (NE + SE) - (NW + SW) and
        // (NE - SE) + (NW - SW), both halves of a pair in one packed instruction
        const float2 P = f2_(rp[c + 1], rp[c - 1]), Q = f2_(rm[c + 1], rm[c - 1]);
        const float2 S = add2_(P, Q), D = sub2_(P, Q);
        const float2 G = fma2_(bc2_(c1), f2_(r0[c + 1] - r0[c - 1], rp[c] - rm[c]),
                               mul2_(bc2_(c2), f2_(S.x - S.y, D.x + D.y)));
        gx = G.x, gy = G.y;
        return;
    }
    const Real ne = rp[c + 1], nw = rp[c - 1], se = rm[c + 1], sw = rm[c - 1];
    gx = c1 * (r0[c + 1] - r0[c - 1]) + c2 * ((ne - nw) + (se - sw));
    gy = c1 * (rp[c] - rm[c]) + c2 * ((ne - se) + (nw - sw));
}

// Loads of one row for the pull: populations of one lattice (plane base pointers `pl`,
// wall rule KIND) at row y and column x, with the wall rules of Sec. 5.1.  Offsets are
// 32-bit element indices; the row part is CTA-uniform.
//   KIND 0: phase field, specular reflection (free slip, no flux through the wall)
//   KIND 1: flow, halfway bounce-back (no slip)
//   KIND 2: energy, anti-bounce-back to the wall temperature where the link crosses the wall
// Values come out in stored units (for FP16 storage: times its scale; wscale multiplies
// the anti-bounce-back wall term accordingly).
template <int KIND, int Q, typename Real, typename Store>
__device__ __forceinline__ void pull_row_(const Store *const *pl, int pitch, int ny, int nx, int y, int x, int xm,
                                          int xp, Real wscale, const Real *__restrict__ twall, Real dTcold, Real *out)
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
        if (KIND == 2 && wall) {
            const Real tw = ey > 0 ? twall[(1 - ex) * nx + x] : dTcold;
            Real t = Real(2.0 * w_<Q>(a)) * tw;
            if constexpr (scaled_<Store>()) t *= wscale;
            v = -v + t;
        }
        out[a] = v;
    }
}

// ---- asynchronous row staging ----------------------------------------------------------
// The population rows a CTA pulls from are copied into shared memory by the bulk-copy (TMA)
// engine, D - 1 output rows ahead of the row being collided: the loads hold no registers
// and each SM keeps several rows of every plane in flight.  Stage k of a CTA serves output
// row y = y0 + k and holds the source rows of f pulled at row y + 3, of h pulled at y + 1
// and of g pulled at y (after the wall rules: the reflected or reversed plane's row at a
// wall), and dp of row y + 1, each over the strip's columns plus a halo on both sides, and
// the row's values of the phase-field reference (StepArgs::rowx).
// Bulk copies move 16-byte aligned spans; columns that wrap around the periodic x edge, or
// lie past the last 16-byte boundary of a row, are copied element by element by all threads
// (cp.async, or plain loads for 2-byte values), and each thread then arrives on the slot's
// mbarrier: a stage is complete when its mbarrier phase is, and every thread waits on it.
__device__ __forceinline__ uint32_t smem_u32_(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init_(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32_(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence_() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx_(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32_(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s_(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32_(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32_(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32_(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the completion of the phase of `bar` with the given parity until the
// %globaltimer deadline t_end (ns); false if it passed: a copy that never lands must not
// hang the GPU.
__device__ __forceinline__ bool mbar_wait_until_(uint64_t *bar, uint32_t parity, uint64_t t_end)
{
    while (!mbar_try_wait_(bar, parity))
        if (globaltimer_() > t_end) return false;
    return true;
}
// the same with a limit of about one second from now
__device__ __forceinline__ bool mbar_wait_(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait_(bar, parity)) return true;
    return mbar_wait_until_(bar, parity, globaltimer_() + 1000000000ull);
}
// one element: cp.async (4 or 8 bytes), or a plain load and store
template <bool ASYNC, typename T>
__device__ __forceinline__ void cp_elem_(T *dst, const T *src)
{
    if constexpr (ASYNC && sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32_(dst)), "l"(src) : "memory");
    else if constexpr (ASYNC && sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32_(dst)), "l"(src) : "memory");
    else
        *dst = *src;
}
// arrive on `bar` once this thread's earlier cp.async copies have landed (counted at init)
__device__ __forceinline__ void cp_arrive_noinc_(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32_(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32_(bar)) : "memory");
}
__device__ __forceinline__ void cp_wait_all_() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename Real, typename Store>
__device__ __forceinline__ Real lds_(const Store *p)
{
    if constexpr (std::is_same<Store, __half>::value) return Real(__half2float(*p));
    else return Real(*p);
}

// Columns per strip: 128.  FP32 storage: five CTAs of 5 warps per SM (72 registers per
// thread, a three-stage ring; measured 1 % faster than four CTAs with a four-stage ring on
// the 8192 x 2048 channel; 256 columns ran 2 % slower).  FP16 storage: six CTAs (64
// registers; its stages are half the size).  FP64 needs ~125-165 registers per thread: two.
template <typename Real> constexpr int march_width() { return 128; }
// Resident CTAs per SM the kernels are built for (registers and shared memory).
template <typename Real, typename Store> constexpr int march_ctas()
{
    return sizeof(Real) == 8 ? 2 : (sizeof(Store) == 2 ? 6 : 5);
}
// The many-channel kernel reads its arguments through a pointer and needs more registers:
// at 72 it spilled and ran the 16-channel sweep 14 % slower than with four CTAs per SM.
template <typename Real> constexpr int batch_ctas() { return sizeof(Real) == 4 ? 4 : 2; }

// Shared-memory geometry of the staging ring (host and device).
template <typename Real, typename Store, int QF, int QT, int TX> struct StageGeo {
    static constexpr int HS = sizeof(Store) == 2 ? 8 : 4;   // halo columns per side, population planes
    static constexpr int HD = 4;                             // halo columns per side, dp plane
    static constexpr int RS = TX + 2 * HS, RD = TX + 2 * HD; // staged row lengths (16-byte multiples)
    static constexpr int NP = QF + QT + 9;                   // population planes per stage: f, h, g
    static constexpr int RXO = NP * RS * (int)sizeof(Store) + RD * (int)sizeof(Real);   // reference values
    static constexpr int BYTES = (RXO + RX_N * (int)sizeof(Real) + 15) / 16 * 16;   // bulk copies need 16 B
    static_assert(RXO % 16 == 0, "the staged reference values need a 16-byte aligned slot");
    static constexpr int RINGS = 8 * (TX + 4) * (int)sizeof(Real) + 16 * (TX + 2) * (int)sizeof(Real);
    // deepest ring that leaves room for march_ctas() CTAs per SM (228 KiB, 1 KiB reserved per CTA)
    static constexpr int BUDGET = 233472 / march_ctas<Real, Store>() - 1024 - 128 - 16 - RINGS;
    static constexpr int D = (4 * BYTES + 128 <= BUDGET) ? 4 : ((3 * BYTES + 128 <= BUDGET) ? 3 : 2);
    static constexpr int DYN = D * BYTES + 128;              // + one mbarrier per slot
};

template <typename Real, typename Store, int QF, int QT, int TX>
__device__ __forceinline__ void march_body(const StepArgs<Real, Store> &A, int seg, int bx, int by)
{
    using R2 = typename Vec2<Real>::T;
    using G = StageGeo<Real, Store, QF, QT, TX>;
    constexpr int PX = TX + 4, SX = TX + 2, NT = TX + 32;
    constexpr int D = G::D, HS = G::HS, HD = G::HD, RS = G::RS, RD = G::RD, NP = G::NP;
    constexpr int CS = 16 / (int)sizeof(Store), CD = 16 / (int)sizeof(Real);   // elements per 16 bytes
    __shared__ Real s_phi[8][PX];   // phi - phi0
    __shared__ R2 s_sp[4][SX];   // (sigma - sigma0, p - p0)
    __shared__ R2 s_n[4][SX];    // unit normal (n_x, n_y - 1)
    __shared__ int s_abort;
    extern __shared__ __align__(128) unsigned char s_dyn[];
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(s_dyn + D * G::BYTES);

    const int nx = A.nx, ny = A.ny, pitch = A.pitch;
    const Phys<Real> &P = A.P;
    // reference-profile row tables for the first rows of a segment (row r at r + 1); the
    // marching loop takes the same values from the staged rows
    const Real *t_dR = A.rtab + (ny + 2) * RT_DR + 1, *t_gref = A.rtab + (ny + 2) * RT_GREF + 1;
    const Real *t_dRlo = A.rtab + (ny + 2) * RT_DRLO + 1;
    const int tid = threadIdx.x;
    const int x0 = bx * TX;
    const int y0 = by * seg;
    const int y1 = min(y0 + seg, ny);
    // Threads 0..TX-1 own the columns x0 + tid (phi, sigma, n, collision and store); the last
    // warp (the edge warp) issues the bulk copies and computes the halo columns: lanes 0..3
    // phi at x0-2, x0-1, x0+TX, x0+TX+1, lanes 0..1 sigma, p and n at x0-1, x0+TX.
    const bool colt = tid < TX;
    const int lane = tid - TX;
    const bool doF = colt || lane < 4, doH = colt || lane < 2;
    const int cf = colt ? tid : (lane < 2 ? lane - 2 : TX + lane - 2);   // column of phi, relative to x0
    const int ch = colt ? tid : (lane == 0 ? -1 : TX);                   // column of sigma and n
    const int x = x0 + tid;
    const bool xin = colt && x < nx;
    const int xf = wrap_(x0 + cf, nx), xh = wrap_(x0 + ch, nx);
    const int xfm = xf == 0 ? nx - 1 : xf - 1, xfp = xf == nx - 1 ? 0 : xf + 1;
    const int xhm = xh == 0 ? nx - 1 : xh - 1, xhp = xh == nx - 1 ? 0 : xh + 1;

    // ---- staging geometry (CTA-uniform) ----
    // staged column j of a population plane is global column sx0 + j (wrapped); the bulk
    // part covers staged columns [boff, boff + bspan), the rest is copied element-wise
    const int sx0 = x0 - HS, dx0 = x0 - HD;
    const int blo = max(sx0, 0), bhi = min(x0 + TX + HS, nx / CS * CS);
    const int bspan = bhi > blo ? bhi - blo : 0, boff = blo - sx0;
    const int dlo = max(dx0, 0), dhi = min(x0 + TX + HD, nx / CD * CD);
    const int dspan = dhi > dlo ? dhi - dlo : 0, doff = dlo - dx0;
    const int nel_s = RS - bspan, nel_d = RD - dspan;          // element-wise columns per plane
    const int n_edge = NP * nel_s + nel_d;
    const bool edge = n_edge > 0;                               // then every thread arrives too
    constexpr bool ASYNC = sizeof(Store) >= 4;
    const uint32_t tx_bytes = uint32_t(NP * bspan * (int)sizeof(Store) + dspan * (int)sizeof(Real) +
                                       RX_N * (int)sizeof(Real));
    auto stage_pop = [&](int sl) { return reinterpret_cast<Store *>(s_dyn + sl * G::BYTES); };
    auto stage_dp = [&](int sl) { return reinterpret_cast<Real *>(s_dyn + sl * G::BYTES + NP * RS * sizeof(Store)); };
    auto stage_rx = [&](int sl) { return reinterpret_cast<const Real *>(s_dyn + sl * G::BYTES + G::RXO); };

    // source row of staged plane p for output row yy: f pulled at yy + 3, h at yy + 1, g at yy
    auto src_row = [&](int p, int yy) -> const Store * {
        int a, r, kind;
        const Store *base;
        if (p < QF) {
            a = p, r = yy + 3, kind = 0, base = A.f_in;
        } else if (p < QF + QT) {
            a = p - QF, r = yy + 1, kind = 2, base = A.h_in;
        } else {
            a = p - QF - QT, r = yy, kind = 1, base = A.g_in;
        }
        const int gy = mirror_row_(r, ny), ey = ey_(a);
        const bool wall = (ey > 0 && gy == 0) || (ey < 0 && gy == ny - 1);
        const int src = wall ? (kind == 0 ? mir_(a) : opp_(a)) : a;
        return base + (long long)src * A.plane + (long long)(wall ? gy : gy - ey) * pitch;
    };
    // Copies of stage `yy` into slot `sl` (every thread calls it; nothing past the segment).
    auto issue = [&](int yy, int sl) {
        if (yy >= y1) return;
        Store *st = stage_pop(sl);
        Real *sd = stage_dp(sl);
        if (!colt) {
            if (lane == 0) mbar_expect_tx_(&s_bar[sl], tx_bytes + A.tx_extra);
            __syncwarp();
            if (lane < NP) {
                if (bspan > 0) bulk_g2s_(st + lane * RS + boff, src_row(lane, yy) + blo, bspan * sizeof(Store), &s_bar[sl]);
            } else if (lane == NP) {
                if (dspan > 0)
                    bulk_g2s_(sd + doff, A.dp_in + (long long)mirror_row_(yy + 1, ny) * pitch + dlo,
                              dspan * sizeof(Real), &s_bar[sl]);
            } else if (lane == NP + 1) {
                bulk_g2s_(const_cast<Real *>(stage_rx(sl)), A.rowx + (long long)yy * RX_N, RX_N * sizeof(Real),
                          &s_bar[sl]);
            }
        }
        if (edge) {
            for (int e = tid; e < n_edge; e += NT) {
                if (e < NP * nel_s) {
                    const int p = e / nel_s, k = e - p * nel_s, j = k < boff ? k : k + bspan;
                    cp_elem_<ASYNC>(st + p * RS + j, src_row(p, yy) + wrap_(sx0 + j, nx));
                } else {
                    const int k = e - NP * nel_s, j = k < doff ? k : k + dspan;
                    cp_elem_<ASYNC>(sd + j, A.dp_in + (long long)mirror_row_(yy + 1, ny) * pitch + wrap_(dx0 + j, nx));
                }
            }
            if constexpr (ASYNC) cp_arrive_noinc_(&s_bar[sl]);
            else mbar_arrive_(&s_bar[sl]);
        }
    };
    // Pulled values of a completed stage at the thread's columns (wall rules of Sec. 5.1), in
    // stored units: with FP16 storage the sums and moments formed from them are rescaled
    // (put_phi_dr, put_sig, keep_f, keep_h, the flow's moments), not each value.
    constexpr bool SCALED = scaled_<Store>();
    auto read_f = [&](int sl, Real *f) {
        const Store *st = stage_pop(sl) + HS + cf;
#pragma unroll
        for (int a = 0; a < QF; ++a) {
            // specular reflection keeps the x shift of the link
            f[a] = lds_<Real, Store>(st + a * RS - ex_(a));
        }
    };
    // WALLS = false: rows away from the walls (no link of this row crosses one)
    auto read_h = [&](auto walls, int sl, int r, Real *h, Real &dp) {
        constexpr bool WALLS = decltype(walls)::value;
        const Store *st = stage_pop(sl) + QF * RS + HS + ch;
        const int gy = mirror_row_(r, ny);
        const bool wb = WALLS && gy == 0, wt = WALLS && gy == ny - 1;
#pragma unroll
        for (int a = 0; a < QT; ++a) {
            const int ex = ex_(a), ey = ey_(a);
            const bool wall = (ey > 0 && wb) || (ey < 0 && wt);
            Real v = lds_<Real, Store>(st + a * RS - (wall ? 0 : ex));
            if (wall) {
                Real t = Real(2.0 * w_<QT>(a)) * (ey > 0 ? A.twall[(1 - ex) * nx + xh] : P.dTcold);
                if constexpr (SCALED) t *= A.sh;
                v = -v + t;
            }
            h[a] = v;
        }
        dp = stage_dp(sl)[HD + ch];
    };
    auto read_g = [&](auto walls, int sl, int y, Real *g) {
        constexpr bool WALLS = decltype(walls)::value;
        const Store *st = stage_pop(sl) + (QF + QT) * RS + HS + tid;
        const bool wb = WALLS && y == 0, wt = WALLS && y == ny - 1;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int ey = ey_(a);
            const bool wall = (ey > 0 && wb) || (ey < 0 && wt);
            g[a] = lds_<Real, Store>(st + a * RS - (wall ? 0 : ex_(a)));
        }
    };
    // Direct loads (first rows of a segment only).
    auto load_f = [&](int r, Real *f) {
        pull_row_<0, QF>(A.fi, pitch, ny, nx, mirror_row_(r, ny), xf, xfm, xfp, A.sf, A.twall, P.dTcold, f);
    };
    auto load_h = [&](int r, Real *h, Real &dp) {
        const int gy = mirror_row_(r, ny);
        pull_row_<2, QT>(A.hi, pitch, ny, nx, gy, xh, xhm, xhp, A.sh, A.twall, P.dTcold, h);
        dp = A.dp_in[gy * pitch + xh];
    };
    // phi - phi0 of row r (ghost rows: of the mirrored row) from the pulled deviations and
    // that row's dR (high and low parts)
    auto put_phi_dr = [&](int r, const Real *f, Real dr, Real drlo) {
        Real dphi = f[0];
#pragma unroll
        for (int a = 1; a < QF; ++a) dphi += f[a];
        if constexpr (SCALED) dphi *= A.isf;
        if constexpr (std::is_same<Real, double>::value) dphi += dr;
        else dphi = (dphi + drlo) + dr;
        s_phi[r & 7][cf + 2] = dphi;
    };
    auto put_phi = [&](int r, const Real *f) {
        const int gy = mirror_row_(r, ny);
        put_phi_dr(r, f, __ldg(t_dR + gy), __ldg(t_dRlo + gy));
    };
    // returns T - T_ref of the pulled populations (of row r itself, not the ghost value)
    auto put_sig = [&](int r, const Real *h, Real dp) -> Real {
        Real dT = h[0];
#pragma unroll
        for (int a = 1; a < QT; ++a) dT += h[a];
        if constexpr (SCALED) dT *= A.ish;
        Real dTs = dT;
        if (r == -1) dTs = Real(2) * A.twall[nx + xh] - dT;   // T_ghost = 2 T_w - T_adjacent
        else if (r == ny) dTs = Real(2) * P.dTcold - dT;
        R2 v;
        v.x = dTs * (P.sigma1 + P.sigma2 * dTs);
        v.y = dp;
        s_sp[r & 3][ch + 1] = v;
        return dT;
    };
    // what the collisions keep of pulled populations: first raw moments of f, and
    // (T - T_ref, first raw moments) of h
    auto keep_f = [&](const Real *f, Real *m) {
        raw_first_<QF>(f, m[0], m[1]);
        if constexpr (SCALED) m[0] *= A.isf, m[1] *= A.isf;
    };
    auto keep_h = [&](const Real *h, Real dT, Real *m) {
        m[0] = dT;
        raw_first_<QT>(h, m[1], m[2]);
        if constexpr (SCALED) m[1] *= A.ish, m[2] *= A.ish;
    };
    // grad phi = grad (phi - phi0) + (0, d_y phi0); the normal as (n_x, n_y - 1)
    auto put_n_g = [&](int r, Real gref) {
        Real gx, gy;
        R2 n;
        grad3_(s_phi[(r - 1) & 7], s_phi[r & 7], s_phi[(r + 1) & 7], ch + 2, gx, gy);
        unit_normal_dev_(gx, gy + gref, P.g2min, n.x, n.y);
        s_n[r & 3][ch + 1] = n;
    };
    auto put_n = [&](int r) { put_n_g(r, __ldg(t_gref + r)); };
    // After a wait gave up: flag the fault, let the copies this CTA started land, return.
    // (k_fail: the stage whose wait gave up; the later stages issued are waited for once
    // more, all within one further second.)  The path assumes that every issued copy, a
    // read of valid global memory, completes in the end; it is exercised with the test hook
    // that makes each stage expect more bytes than it copies.
    auto fail = [&](int k_fail, int k_last) {
        cp_wait_all_();
        if (tid == 0) {
            if (A.fault) atomicOr(A.fault, 1u);
            const uint64_t t_end = globaltimer_() + 1000000000ull;
            for (int k = k_fail + 1; k <= k_last; ++k)
                if (!mbar_wait_until_(&s_bar[k % D], uint32_t((k / D) & 1), t_end)) break;
        }
    };

    // ---- prologue: barriers; stages y0 .. y0+D-2 in flight; phi rows y0-2 .. y0+2,
    // sigma/p rows y0-1, y0 and normals y0-1, y0 from direct loads ----
    if (tid == 0) {
        for (int k = 0; k < D; ++k) mbar_init_(&s_bar[k], edge ? NT + 1 : 1);
        s_abort = 0;
        mbar_init_fence_();
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < D - 1; ++k) issue(y0 + k, k);
    // first raw moments of f pulled at rows y0 .. y0 + 2 and (T - T_ref, first raw
    // moments) of h pulled at row y0: all the collisions need of those populations
    Real fm0[2], fm1[2], fm2[2], hm0[3];
    if (doF) {
        Real t[QF];
        load_f(y0 - 2, t);
        put_phi(y0 - 2, t);
        load_f(y0 - 1, t);
        put_phi(y0 - 1, t);
        load_f(y0, t);
        put_phi(y0, t);
        keep_f(t, fm0);
        load_f(y0 + 1, t);
        put_phi(y0 + 1, t);
        keep_f(t, fm1);
        load_f(y0 + 2, t);
        put_phi(y0 + 2, t);
        keep_f(t, fm2);
    }
    if (doH) {
        Real t[QT], dp;
        load_h(y0 - 1, t, dp);
        put_sig(y0 - 1, t, dp);
        load_h(y0, t, dp);
        keep_h(t, put_sig(y0, t, dp), hm0);
    }
    __syncthreads();
    if (doH) {
        put_n(y0 - 1);
        put_n(y0);
    }

    const Real c2 = Real(1.0 / 3.0), hf = Real(0.5);
    int sl = 0;          // slot of the stage of row y
    uint32_t par = 0;    // its mbarrier phase parity
    // One barrier per row: before it, phi of row y + 3, sigma and p of row y + 1 and the
    // normals of row y + 1 (from phi rows y .. y + 2, complete since the previous barrier);
    // after it, row y collides.  The rings are deep enough that these writes never touch
    // rows the previous row's collision may still be reading.
    for (int y = y0; y < y1; ++y) {
        Real fm3[2], hm1[3], g[9];
        if (!mbar_wait_(&s_bar[sl], par)) s_abort = 1;
        Real rx[RX_N];   // this row's reference values, read before the slot is refilled
        load_rowref_(stage_rx(sl), rx);
        if (doF) {
            Real t[QF];
            read_f(sl, t);
            put_phi_dr(y + 3, t, rx[RX_DR3], rx[RX_DR3LO]);
            keep_f(t, fm3);
        }
        if (y >= 1 && y <= ny - 3) {   // rows y and y + 1 are clear of the walls
            if (doH) {
                Real t[QT], dp;
                read_h(std::false_type(), sl, y + 1, t, dp);
                keep_h(t, put_sig(y + 1, t, dp), hm1);
                put_n_g(y + 1, rx[RX_GREF1]);
            }
            if (colt) read_g(std::false_type(), sl, y, g);
        } else {
            if (doH) {
                Real t[QT], dp;
                read_h(std::true_type(), sl, y + 1, t, dp);
                keep_h(t, put_sig(y + 1, t, dp), hm1);
                put_n_g(y + 1, rx[RX_GREF1]);
            }
            if (colt) read_g(std::true_type(), sl, y, g);
        }
        const Real phi_ref = rx[RX_PHI0], th0 = rx[RX_TH0], c01 = rx[RX_C01], gref = rx[RX_GREF];
        // refill the slot read one row ago (every thread is past its reads) with row y + D - 1
        issue(y + D - 1, sl == 0 ? D - 1 : sl - 1);
        if (++sl == D) {
            sl = 0;
            par ^= 1u;
        }
        __syncthreads();
        if (s_abort) {
            fail(y - y0, min(y + D - 1, y1 - 1) - y0);
            return;
        }
        if (xin) {
            const int c = tid + 2, s = tid + 1;
            const Real *pm = s_phi[(y - 1) & 7], *p0 = s_phi[y & 7], *pp = s_phi[(y + 1) & 7];
            const Real dphi = p0[c];
            const Real phi = phi_ref + dphi;
            Real gpx, gpy;
            grad3_(pm, p0, pp, c, gpx, gpy);
            gpy += gref;
            const Real g2 = gpx * gpx + gpy * gpy;
            const R2 *nm = s_n[(y - 1) & 3], *n0 = s_n[y & 3], *np = s_n[(y + 1) & 3];
            const R2 *qm = s_sp[(y - 1) & 3], *q0 = s_sp[y & 3], *qp = s_sp[(y + 1) & 3];
            const R2 nC = n0[s], nE = n0[s + 1], nW = n0[s - 1], nN = np[s], nS = nm[s];
            const R2 nNE = np[s + 1], nNW = np[s - 1], nSE = nm[s + 1], nSW = nm[s - 1];
            const Real c1 = Real(1.0 / 3.0), cd = Real(1.0 / 12.0);
            const R2 qE = q0[s + 1], qW = q0[s - 1], qN = qp[s], qS = qm[s];
            const R2 qNE = qp[s + 1], qNW = qp[s - 1], qSE = qm[s + 1], qSW = qm[s - 1];
            Real divn, dsx, dsy, dpx, dpy;
            if constexpr (std::is_same<Real, float>::value) {
                // the same stencils with the (n_x, n_y) and (sigma, p) halves paired; the
                // diagonal terms of div n summed as (NE - SW) +- (SE - NW)
                const float2 T1 = sub2_(nNE, nSW), T2 = sub2_(nSE, nNW);
                divn = c1 * ((nE.x - nW.x) + (nN.y - nS.y)) + cd * ((T1.x + T2.x) + (T1.y - T2.y));
                const float2 X = fma2_(bc2_(c1), sub2_(qE, qW), mul2_(bc2_(cd), add2_(sub2_(qNE, qNW), sub2_(qSE, qSW))));
                const float2 Y = fma2_(bc2_(c1), sub2_(qN, qS), mul2_(bc2_(cd), add2_(sub2_(qNE, qSE), sub2_(qNW, qSW))));
                dsx = X.x, dpx = X.y, dsy = Y.x, dpy = Y.y;
            } else {
                divn = c1 * (nE.x - nW.x) + cd * ((nNE.x - nNW.x) + (nSE.x - nSW.x)) + c1 * (nN.y - nS.y) +
                       cd * ((nNE.y - nSE.y) + (nNW.y - nSW.y));
                dsx = c1 * (qE.x - qW.x) + cd * ((qNE.x - qNW.x) + (qSE.x - qSW.x));
                dsy = c1 * (qN.x - qS.x) + cd * ((qNE.x - qSE.x) + (qNW.x - qSW.x));
                dpx = c1 * (qE.y - qW.y) + cd * ((qNE.y - qNW.y) + (qSE.y - qSW.y));
                dpy = c1 * (qN.y - qS.y) + cd * ((qNE.y - qSE.y) + (qNW.y - qSW.y));
            }
            const Real nxv = nC.x, nyv = Real(1) + nC.y;
            const Real dT = hm0[0];
            const Real sigma = P.sigma0 + dT * (P.sigma1 + P.sigma2 * dT);
            const Real Fsx = P.csf * (-sigma * g2 * divn * nxv + g2 * ((Real(1) - nxv * nxv) * dsx - nxv * nyv * dsy));
            const Real Fsy = P.csf * (-sigma * g2 * divn * nyv + g2 * ((Real(1) - nyv * nyv) * dsy - nxv * nyv * dsx));
            const Real Ftx = Fsx + P.Fx, Fty = Fsy + P.Fy;
            const Real Fpx = -dpx + c2 * P.drho * gpx, Fpy = -dpy + c2 * P.drho * gpy;
            const Real rho = P.rhoA + phi * P.drho;
            const Real irho = rcp_(rho);
            Real s0, sx, sy, r20, r02, r11;
            flow_raw_moments_(g, s0, sx, sy, r20, r02, r11);
            if constexpr (SCALED) s0 *= A.isg, sx *= A.isg, sy *= A.isg, r20 *= A.isg, r02 *= A.isg, r11 *= A.isg;
            const Real irc2 = Real(3) * irho;
            const Real ux = (sx + hf * c2 * Ftx) * irc2;
            const Real uy = (sy + hf * c2 * Fty) * irc2;
            const Real dp = s0 + hf * (Fpx * ux + Fpy * uy);
            const Real om_nu = rcp_(Real(3) * (P.muA + phi * P.dmu) * irho + hf);
            const Real om_T = rcp_(Real(3) * (P.kA + phi * P.dk) * irho + hf);
            // theta(phi) - theta(phi0) = (4 / W) dphi (1 - 2 phi0 - dphi)
            const Real dth = P.W4 * dphi * (Real(1) - Real(2) * phi_ref - dphi);
            Real fo[QF], ho[QT];
            // (FP16 storage: the results come out in stored units)
            collide_phase_dev_<QF, Real, SCALED>(fo, fm0[0], fm0[1], dphi, phi, ux, uy, nxv, nC.y, th0, dth, c01,
                                                 P.Mphi, P.omega_phi, A.sf);
            collide_flow_<Real, SCALED>(g, rho, dp, ux, uy, Fpx, Fpy, Ftx, Fty, om_nu, s0, sx, sy, r20, r02, r11, A.sg);
            collide_energy_<QT, Real, SCALED>(ho, hm0[1], hm0[2], dT, ux, uy, P.T_ref, om_T, A.sh);
            const int o = y * pitch + x;
            // one unsigned 32-bit byte offset from every plane's base (measured 2 % faster than
            // plane base + element index)
            const uint32_t ob = uint32_t(o) * uint32_t(sizeof(Store));
            auto at = [&](Store *base) { return reinterpret_cast<Store *>(reinterpret_cast<char *>(base) + ob); };
#pragma unroll
            for (int a = 0; a < QF; ++a) {
                st_(at(A.fo[a]), fo[a]);
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                st_(at(A.go[a]), g[a]);
            }
#pragma unroll
            for (int a = 0; a < QT; ++a) {
                st_(at(A.ho[a]), ho[a]);
            }
            A.dp_out[o] = dp;
            if (A.macro) {
                const long long N = (long long)nx * ny, m = (long long)y * nx + x;
                A.macro[m] = A.phi0[y] + double(dphi);
                A.macro[N + m] = double(ux);
                A.macro[2 * N + m] = double(uy);
                A.macro[3 * N + m] = double(P.T_ref) + double(dT);
                A.macro[4 * N + m] = double(dp);
            }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            fm0[a] = fm1[a];
            fm1[a] = fm2[a];
            fm2[a] = fm3[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) hm0[a] = hm1[a];
    }
}

template <typename Real, typename Store, int QF, int QT, int TX>
__global__ void __launch_bounds__(TX + 32, march_ctas<Real, Store>()) march_kernel(const StepArgs<Real, Store> A, int seg)
{
    march_body<Real, Store, QF, QT, TX>(A, seg, blockIdx.x, blockIdx.y);
}

// Many channels of uneven size in one launch: CTA i works on strip ctas[i].y, segment
// ctas[i].z of case ctas[i].x, with that case's arguments; cases whose active flag is 0
// (converged) are skipped.
template <typename Real, typename Store, int QF, int QT, int TX>
__global__ void __launch_bounds__(TX + 32, batch_ctas<Real>()) batch_kernel(const StepArgs<Real, Store> *__restrict__ cases,
                                                       const int4 *__restrict__ ctas, const int *__restrict__ active,
                                                       int seg)
{
    const int4 t = ctas[blockIdx.x];
    if (!active[t.x]) return;
    march_body<Real, Store, QF, QT, TX>(cases[t.x], seg, t.y, t.z);
}


template <typename Real, typename Store, int QF, int QT>
int step_strip_width()
{
    return march_width<Real>();
}

// Dynamic shared memory of the step kernels (the staging ring); the attribute that allows
// it is set once per kernel instance, with the carveout at its shared-memory maximum.
template <typename Real, typename Store, int QF, int QT>
static int prepare_kernels()
{
    constexpr int TX = march_width<Real>();
    constexpr int dyn = StageGeo<Real, Store, QF, QT, TX>::DYN;
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(march_kernel<Real, Store, QF, QT, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaFuncSetAttribute(batch_kernel<Real, Store, QF, QT, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaFuncSetAttribute(march_kernel<Real, Store, QF, QT, TX>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
        cudaFuncSetAttribute(batch_kernel<Real, Store, QF, QT, TX>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
        done = true;
    }
    return dyn;
}

template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_batch(const StepArgs<Real, Store> *cases, const int4 *ctas, int n_ctas, const int *active, int seg,
                         cudaStream_t s)
{
    constexpr int TX = march_width<Real>();
    const int dyn = prepare_kernels<Real, Store, QF, QT>();
    batch_kernel<Real, Store, QF, QT, TX><<<n_ctas, TX + 32, dyn, s>>>(cases, ctas, active, seg);
    return cudaGetLastError();
}

template <typename Real, typename Store, int QF, int QT>
int resident_ctas()
{
    constexpr int TX = march_width<Real>();
    const int dyn = prepare_kernels<Real, Store, QF, QT>();
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<Real, Store, QF, QT, TX>, TX + 32, dyn);
    return sms * (per_sm > 0 ? per_sm : 1);
}

// Segment length: the one that minimises the estimated step time, waves of resident CTAs
// times (rows per segment + the ~6 start-up rows each segment re-derives), preferring longer
// segments on ties.  Small grids get short segments (more CTAs in one wave); large grids
// whole waves.  Segments are at least 8 rows.
static int choose_segment(int strips, int ny, int slots)
{
    int best = ny;
    long long best_cost = -1;
    for (int nseg = 1; nseg <= (ny + 7) / 8; ++nseg) {
        const int seg = (ny + nseg - 1) / nseg;
        const int used = (ny + seg - 1) / seg;          // segments actually launched
        const long long ctas = (long long)strips * used;
        const long long waves = (ctas + slots - 1) / slots;
        const long long cost = waves * (seg + 6);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = seg;
        }
    }
    return best;
}

// resident CTAs of the step kernel on the device (per template instance)
template <typename Real, typename Store, int QF, int QT>
static int march_slots()
{
    constexpr int TX = march_width<Real>();
    const int dyn = prepare_kernels<Real, Store, QF, QT>();
    static int slots = 0;
    if (slots == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_kernel<Real, Store, QF, QT, TX>, TX + 32, dyn);
        slots = sms * (per_sm > 0 ? per_sm : 1);
    }
    return slots;
}

template <typename Real, typename Store, int QF, int QT>
int auto_segment(int nx, int ny)
{
    constexpr int TX = march_width<Real>();
    return choose_segment((nx + TX - 1) / TX, ny, march_slots<Real, Store, QF, QT>());
}

template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_step(const StepArgs<Real, Store> &A, cudaStream_t s, int seg_rows)
{
    constexpr int TX = march_width<Real>();
    const int dyn = prepare_kernels<Real, Store, QF, QT>();
    const int seg = seg_rows > 0 ? (seg_rows < A.ny ? seg_rows : A.ny) : auto_segment<Real, Store, QF, QT>(A.nx, A.ny);
    dim3 grid((A.nx + TX - 1) / TX, (A.ny + seg - 1) / seg);
    march_kernel<Real, Store, QF, QT, TX><<<grid, TX + 32, dyn, s>>>(A, seg);
    return cudaGetLastError();
}

#define LBM_INST(R, S, QF, QT)                                                                              \
    template cudaError_t launch_step<R, S, QF, QT>(const StepArgs<R, S> &, cudaStream_t, int);             \
    template cudaError_t launch_batch<R, S, QF, QT>(const StepArgs<R, S> *, const int4 *, int, const int *, \
                                                    int, cudaStream_t);                                   \
    template int step_strip_width<R, S, QF, QT>();                                                         \
    template int auto_segment<R, S, QF, QT>(int, int);                                                     \
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
