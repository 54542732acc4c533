// Lattice-Boltzmann stream-collide: one thread per node, fused pull-streaming, diffuse
// kinetic walls, regularised BGK collision and Hermite body force (Sec. 2 "ingredients":
// kinetic boundary conditions, higher-order lattice, regularisation; Sec. 3.1, Eq. tau).
//
// Populations are stored f[q][y][x] (x across the channel, fastest), so consecutive threads
// pull consecutive addresses for every q; each node reads its 39 (or 19) populations once
// and writes them once (312 B per node-update in FP32 for D3Q39).
//
// Collision, in the moment space of the Hermite expansion (exact on the quadrature):
//   rho = sum f, j = sum f xi, Pi = sum f xi xi, Qm = sum f xi xi xi (D3Q39),
//   u = (j + rho g / 2) / rho,
//   non-equilibrium Hermite coefficients a1 = -rho g / 2, a2 = Pi - rho(uu + I),
//   a3 = Qm - rho(uuu + sym(u I)) - sym(a1 I),
//   f' = f_eq + (1 - 1/tau) w [a1.xi + a2:H2/2 + a3:H3/6] + (1 - 1/(2 tau)) F,
//   f_eq = w rho [1 + xi.u + ((xi.u)^2 - u^2)/2 + (xi.u)((xi.u)^2 - 3u^2)/6],
//   F = w [rho g.xi + rho (g u + u g):H2/2 + rho sym(g u u):H3/6].
// All three parts are Hermite series, so f' = w [A0 + A1.xi + A2:H2/2 + A3:H3/6] with
//   A0 = rho, A1 = rho u + om a1 + of rho g, A2 = rho uu + om a2 + of rho (gu + ug),
//   A3 = rho uuu + om a3 + of rho sym(guu)      (om = 1 - 1/tau, of = 1 - 1/(2 tau)).
// The populations come in pairs xi, -xi; with s = f(xi) + f(-xi) and d = f(xi) - f(-xi) the
// even moments take s and the odd ones d, and f'(+-xi) = w (E +- O) with E the even part
// (A0, A2) and O the odd part (A1, A3) of the series. Every lattice constant is a
// compile-time value, so terms with zero speed components vanish at compile time.
#include <cstring>
#include <utility>

#include "hyb_internal.cuh"

namespace hyb {

namespace {

template <class F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <class LAT>
__host__ __device__ constexpr int E(int a, int i) {
    return LatTab<LAT>::e(a, i);
}
template <class LAT>
__host__ __device__ constexpr double W(int a) {
    return LatTab<LAT>::w(a);
}
// Index of the population with the opposite speed.
template <class LAT>
__host__ __device__ constexpr int opp(int a) {
    for (int b = 0; b < LAT::Q; ++b)
        if (E<LAT>(b, 0) == -E<LAT>(a, 0) && E<LAT>(b, 1) == -E<LAT>(a, 1) &&
            E<LAT>(b, 2) == -E<LAT>(a, 2))
            return b;
    return -1;
}

__device__ __forceinline__ int wrap_y(int v, int ny) {
    while (v < 0) v += ny;
    while (v >= ny) v -= ny;
    return v;
}

// Pull streaming of node (x, y[, z]): fs[q] = f[q](x - e_q), periodic in y (and in z in 3D);
// sources behind a wall take the wall Maxwellian with the wall density of the streamwise row
// (y, z) (the mass leaving through that wall, re-emitted at rest).
template <typename Real, class LAT, bool Z3 = false>
__device__ __forceinline__ void pull_node(const Real* __restrict__ src, int x, int y, int nx, int ny,
                                          int64_t nn, Real (&fs)[LAT::Q], int z = 0, int nz = 1) {
    constexpr int Q = LAT::Q;
    // Row offsets y' * nx of the pull sources y' = y - ey (periodic), ey = -MAXV..MAXV, and in
    // 3D the layer offsets z' nx ny of z' = z - ez (periodic).
    constexpr int MV = LAT::MAXV;
    int rowoff[2 * MV + 1];
#pragma unroll
    for (int i = 0; i < 2 * MV + 1; ++i) rowoff[i] = wrap_y(y - (i - MV), ny) * nx;
    int64_t layoff[Z3 ? 2 * MV + 1 : 1];
    layoff[0] = 0;
    if constexpr (Z3) {
#pragma unroll
        for (int i = 0; i < 2 * MV + 1; ++i) layoff[i] = (int64_t)wrap_y(z - (i - MV), nz) * nx * ny;
    }
    (void)nz;

    Real rhoL = (Real)0, rhoR = (Real)0;
    if (x < MV || x >= nx - MV) {
        Real ml = (Real)0, mr = (Real)0;
        static_for<Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
            const Real* __restrict__ sq =
                src + (int64_t)q * nn + rowoff[ey + MV] + (Z3 ? layoff[Z3 ? ez + MV : 0] : 0);
            if constexpr (ex < 0) {
#pragma unroll
                for (int i = 0; i < -ex; ++i) ml += sq[i];
            }
            if constexpr (ex > 0) {
#pragma unroll
                for (int i = 0; i < ex; ++i) mr += sq[nx - ex + i];
            }
        });
        constexpr double inv_flux = 1.0 / wall_flux_norm<LAT>();
        rhoL = ml * (Real)inv_flux;
        rhoR = mr * (Real)inv_flux;
    }

    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
        const Real* __restrict__ sq = src + (int64_t)q * nn + (Z3 ? layoff[Z3 ? ez + MV : 0] : 0);
        const int sx = x - ex;
        const int off = rowoff[ey + MV] + sx;
        if constexpr (ex > 0)
            fs[q] = sx < 0 ? (Real)W<LAT>(q) * rhoL : sq[off];
        else if constexpr (ex < 0)
            fs[q] = sx >= nx ? (Real)W<LAT>(q) * rhoR : sq[off];
        else
            fs[q] = sq[off];
    });
}

// Raw moments of the streamed populations from the pair sums s and differences d:
// rho, j, P (xx xy xz yy yz zz) and, for order 3, Q3 (xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz).
template <typename Real, class LAT>
__device__ __forceinline__ void node_moments(const Real (&fs)[LAT::Q], Real& rho, Real& jx, Real& jy,
                                             Real& jz, Real (&pm)[6], Real (&q3)[10]) {
    constexpr int Q = LAT::Q;
    constexpr double R = lat_r<LAT>();
    rho = fs[0];
    jx = jy = jz = (Real)0;
#pragma unroll
    for (int k = 0; k < 6; ++k) pm[k] = (Real)0;
#pragma unroll
    for (int k = 0; k < 10; ++k) q3[k] = (Real)0;
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int p = opp<LAT>(q);
        if constexpr (q != 0 && q < p) {
            constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
            const Real sm = fs[q] + fs[p], df = fs[q] - fs[p];
            rho += sm;
            if constexpr (ex != 0) jx += df * (Real)(R * ex);
            if constexpr (ey != 0) jy += df * (Real)(R * ey);
            if constexpr (ez != 0) jz += df * (Real)(R * ez);
            if constexpr (ex != 0) pm[0] += sm * (Real)(R * R * ex * ex);
            if constexpr (ex * ey != 0) pm[1] += sm * (Real)(R * R * ex * ey);
            if constexpr (ex * ez != 0) pm[2] += sm * (Real)(R * R * ex * ez);
            if constexpr (ey != 0) pm[3] += sm * (Real)(R * R * ey * ey);
            if constexpr (ey * ez != 0) pm[4] += sm * (Real)(R * R * ey * ez);
            if constexpr (ez != 0) pm[5] += sm * (Real)(R * R * ez * ez);
            if constexpr (LAT::ORDER >= 3) {
                constexpr double R3 = R * R * R;
                if constexpr (ex != 0) q3[0] += df * (Real)(R3 * ex * ex * ex);
                if constexpr (ex * ey != 0) q3[1] += df * (Real)(R3 * ex * ex * ey);
                if constexpr (ex * ez != 0) q3[2] += df * (Real)(R3 * ex * ex * ez);
                if constexpr (ex * ey != 0) q3[3] += df * (Real)(R3 * ex * ey * ey);
                if constexpr (ex * ey * ez != 0) q3[4] += df * (Real)(R3 * ex * ey * ez);
                if constexpr (ex * ez != 0) q3[5] += df * (Real)(R3 * ex * ez * ez);
                if constexpr (ey != 0) q3[6] += df * (Real)(R3 * ey * ey * ey);
                if constexpr (ey * ez != 0) q3[7] += df * (Real)(R3 * ey * ey * ez);
                if constexpr (ey * ez != 0) q3[8] += df * (Real)(R3 * ey * ez * ez);
                if constexpr (ez != 0) q3[9] += df * (Real)(R3 * ez * ez * ez);
            }
        }
    });
}

// One node of one context; PARAM: the force increment and relaxation time of the node come
// from the per-node arrays. BGK: the unregularised collision of the proof-of-concept hybrid
// (Sec. 4), f' = (1 - om) f_eq + om f + of F: the series then carries (1 - om) times the
// equilibrium coefficients plus the force, and om f is added per population.
template <typename Real, class LAT, bool PARAM, bool BGK = false, bool Z3 = false>
__device__ __forceinline__ void lbm_node(const LbmArgs<Real>& a, const int64_t node) {
    constexpr int Q = LAT::Q;
    constexpr double R = lat_r<LAT>();
    const int nx = a.nx, ny = a.ny;
    const int64_t nn = a.nnodes;

    Real fs[Q];
    if constexpr (Z3) {  // node (z ny + y) nx + x
        const int64_t row = node / nx;
        pull_node<Real, LAT, true>(a.src, (int)(node % nx), (int)(row % ny), nx, ny, nn, fs,
                                   (int)(row / ny), a.nz);
    } else {
        pull_node<Real, LAT>(a.src, (int)(node % nx), (int)(node / nx), nx, ny, nn, fs);
    }
    Real rho, jx, jy, jz, pm[6], q3[10];
    node_moments<Real, LAT>(fs, rho, jx, jy, jz, pm, q3);
    const Real pxx = pm[0], pxy = pm[1], pxz = pm[2], pyy = pm[3], pyz = pm[4], pzz = pm[5];

    Real gy = a.g_step, om = a.om, of = a.of;
    if constexpr (PARAM) {  // per-node values where given (a Kn profile gives tau only)
        if (a.g_node) gy = a.g_node[node];
        if (a.tau_node) {
            const Real tau = a.tau_node[node];
            om = (Real)1 - (Real)1 / tau;
            of = (Real)1 - (Real)0.5 / tau;
        }
    }
    const Real inv_rho = (Real)1 / rho;
    const Real ux = jx * inv_rho, uy = (jy + (Real)0.5 * rho * gy) * inv_rho, uz = jz * inv_rho;
    const Real a1y = (Real)-0.5 * rho * gy;  // H1 part of f_neq
    const Real rg = rho * gy;
    // combined coefficients of the post-collision series (BGK: the equilibrium weighted by
    // ke = 1 - om and no projected non-equilibrium part, om_r = 0)
    const Real ke = BGK ? (Real)1 - om : (Real)1;
    const Real omr = BGK ? (Real)0 : om;
    const Real rk = ke * rho;
    const Real A0 = rk;
    const Real A1x = rk * ux, A1y = rk * uy + omr * a1y + of * rg, A1z = rk * uz;
    // a2 = Pi - rho (uu + I); A2 = rho uu + om a2 + of rho (gu + ug)
    const Real Axx = rk * ux * ux + omr * (pxx - rho * (ux * ux + (Real)1));
    const Real Ayy = rk * uy * uy + omr * (pyy - rho * (uy * uy + (Real)1)) + of * (Real)2 * rg * uy;
    const Real Azz = rk * uz * uz + omr * (pzz - rho * (uz * uz + (Real)1));
    const Real Axy = rk * ux * uy + omr * (pxy - rho * ux * uy) + of * rg * ux;
    const Real Axz = rk * ux * uz + omr * (pxz - rho * ux * uz);
    const Real Ayz = rk * uy * uz + omr * (pyz - rho * uy * uz) + of * rg * uz;
    const Real tr2 = Axx + Ayy + Azz;
    const Real E0 = A0 - (Real)0.5 * tr2;  // even part without the xi xi terms
    // a3 = Qm - rho(uuu + sym(u I)) - sym(a1 I); A3 = rho uuu + om a3 + of rho sym(guu)
    Real B3[10];
    Real t3x = 0, t3y = 0, t3z = 0;
    if constexpr (LAT::ORDER >= 3) {
        const Real c0 = q3[0] - rho * (ux * ux * ux + (Real)3 * ux);
        const Real c1 = q3[1] - rho * (ux * ux * uy + uy) - a1y;
        const Real c2 = q3[2] - rho * (ux * ux * uz + uz);
        const Real c3 = q3[3] - rho * (ux * uy * uy + ux);
        const Real c4 = q3[4] - rho * (ux * uy * uz);
        const Real c5 = q3[5] - rho * (ux * uz * uz + ux);
        const Real c6 = q3[6] - rho * (uy * uy * uy + (Real)3 * uy) - (Real)3 * a1y;
        const Real c7 = q3[7] - rho * (uy * uy * uz + uz);
        const Real c8 = q3[8] - rho * (uy * uz * uz + uy) - a1y;
        const Real c9 = q3[9] - rho * (uz * uz * uz + (Real)3 * uz);
        B3[0] = rk * ux * ux * ux + omr * c0;
        B3[1] = rk * ux * ux * uy + omr * c1 + of * rg * ux * ux;
        B3[2] = rk * ux * ux * uz + omr * c2;
        B3[3] = rk * ux * uy * uy + omr * c3 + of * (Real)2 * rg * ux * uy;
        B3[4] = rk * ux * uy * uz + omr * c4 + of * rg * ux * uz;
        B3[5] = rk * ux * uz * uz + omr * c5;
        B3[6] = rk * uy * uy * uy + omr * c6 + of * (Real)3 * rg * uy * uy;
        B3[7] = rk * uy * uy * uz + omr * c7 + of * (Real)2 * rg * uy * uz;
        B3[8] = rk * uy * uz * uz + omr * c8 + of * rg * uz * uz;
        B3[9] = rk * uz * uz * uz + omr * c9;
        t3x = B3[0] + B3[3] + B3[5];
        t3y = B3[1] + B3[6] + B3[8];
        t3z = B3[2] + B3[7] + B3[9];
    }
    Real* __restrict__ dst = a.dst + node;

    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int p = opp<LAT>(q);
        if constexpr (q == 0) {
            if constexpr (BGK)
                dst[0] = (Real)W<LAT>(0) * E0 + om * fs[0];
            else
                dst[0] = (Real)W<LAT>(0) * E0;
        } else if constexpr (q < p) {
            constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
            constexpr double X = R * ex, Y = R * ey, Z = R * ez;
            // even part: A0 + A2:H2/2
            Real h2 = (Real)0;
            if constexpr (ex != 0) h2 += (Real)(0.5 * X * X) * Axx;
            if constexpr (ey != 0) h2 += (Real)(0.5 * Y * Y) * Ayy;
            if constexpr (ez != 0) h2 += (Real)(0.5 * Z * Z) * Azz;
            if constexpr (ex * ey != 0) h2 += (Real)(X * Y) * Axy;
            if constexpr (ex * ez != 0) h2 += (Real)(X * Z) * Axz;
            if constexpr (ey * ez != 0) h2 += (Real)(Y * Z) * Ayz;
            const Real ev = E0 + h2;
            // odd part: A1.xi + A3:H3/6
            Real od = (Real)0;
            if constexpr (ex != 0) od += (Real)X * A1x;
            if constexpr (ey != 0) od += (Real)Y * A1y;
            if constexpr (ez != 0) od += (Real)Z * A1z;
            if constexpr (LAT::ORDER >= 3) {
                constexpr double s6 = 1.0 / 6.0;
                if constexpr (ex != 0) od += (Real)(s6 * X * X * X) * B3[0] - (Real)(0.5 * X) * t3x;
                if constexpr (ex * ey != 0) od += (Real)(0.5 * X * X * Y) * B3[1];
                if constexpr (ex * ez != 0) od += (Real)(0.5 * X * X * Z) * B3[2];
                if constexpr (ex * ey != 0) od += (Real)(0.5 * X * Y * Y) * B3[3];
                if constexpr (ex * ey * ez != 0) od += (Real)(X * Y * Z) * B3[4];
                if constexpr (ex * ez != 0) od += (Real)(0.5 * X * Z * Z) * B3[5];
                if constexpr (ey != 0) od += (Real)(s6 * Y * Y * Y) * B3[6] - (Real)(0.5 * Y) * t3y;
                if constexpr (ey * ez != 0) od += (Real)(0.5 * Y * Y * Z) * B3[7];
                if constexpr (ey * ez != 0) od += (Real)(0.5 * Y * Z * Z) * B3[8];
                if constexpr (ez != 0) od += (Real)(s6 * Z * Z * Z) * B3[9] - (Real)(0.5 * Z) * t3z;
            }
            constexpr double wq = W<LAT>(q);
            if constexpr (BGK) {
                dst[(int64_t)q * nn] = (Real)wq * (ev + od) + om * fs[q];
                dst[(int64_t)p * nn] = (Real)wq * (ev - od) + om * fs[p];
            } else {
                dst[(int64_t)q * nn] = (Real)wq * (ev + od);
                dst[(int64_t)p * nn] = (Real)wq * (ev - od);
            }
        }
    });
}

// One thread per node (the nodes of all replicas in the batch form); BGK selects the
// unregularised collision (one instantiation per collision keeps each one's registers).
template <typename Real, class LAT, bool BATCH, bool BGK = false, bool PARAM = false, bool Z3 = false>
__global__ void __launch_bounds__(128) k_lbm(Launch<LbmArgs<Real>> L) {
    pdl_begin();
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= L.total) return;
    if constexpr (BATCH) {
        const int r = replica_of(L.pre, L.nrep, u);
        lbm_node<Real, LAT, PARAM, BGK>(L.tab[r], u - L.pre[r]);
    } else {
        lbm_node<Real, LAT, PARAM, BGK, Z3>(L.one, u);
    }
}

// One thread per node, with per-node force increment and relaxation time.
template <typename Real, class LAT, bool BGK, bool Z3 = false>
__global__ void __launch_bounds__(128) k_lbm_param(LbmArgs<Real> a) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u < a.nnodes) lbm_node<Real, LAT, true, BGK, Z3>(a, u);
}

// ---------------------------------------------------------------------------------------
// Adjoint of one LBM step with per-node force increment g and relaxation time tau. With
// f_{t+1}(x) = C(fs(x); g_x, tau_x) and fs = the pull streaming (with the wall densities) of
// f_t, the adjoint lam_t = dL/df_t is P^T mu, mu(x) = (dC/dfs)^T lam_{t+1}(x), and
// dL/dg_x, dL/dtau_x gather (dC/dg)^T lam_{t+1}(x) and (dC/dtau)^T lam_{t+1}(x) over the
// steps. mu is formed in reverse through the same intermediates as the forward node:
// populations -> combined coefficients (A0, A1, A2, B3) -> (rho, u, P, Q3, g, om, of) ->
// raw moments -> streamed populations. P^T is a permutation: mu_q(x) goes to
// lam_t[q](x - e_q), except for sources behind a wall, whose mu feeds the wall density of
// the row (summed in `wall` and spread over the populations leaving through that wall by
// the last block of k_lbm_adj).

// Third-order terms of B3[k] (k = xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz):
//   B3[k] = rho M_k(u) + om (Q3_k - rho (M_k + L_k(u)) - kap_k a1y) + of rho g f_k(u),
// M_k = u_i u_j u_k, L_k the sym(u I) terms, kap_k the sym(a1 I) multiplicity of a1y,
// f_k the force terms of sym(g u u) / rho g. Returns M, L, f and their u-gradients.
template <typename Real>
__device__ __forceinline__ void b3_terms(int k, Real ux, Real uy, Real uz, Real& M, Real (&dM)[3],
                                         Real& Lk, Real (&dL)[3], Real& kap, Real& fk,
                                         Real (&df)[3]) {
    constexpr int I[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                              {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
    const Real u[3] = {ux, uy, uz};
    const int i = I[k][0], j = I[k][1], l = I[k][2];
    M = u[i] * u[j] * u[l];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Real d = (Real)0;
        if (i == c) d += u[j] * u[l];
        if (j == c) d += u[i] * u[l];
        if (l == c) d += u[i] * u[j];
        dM[c] = d;
        dL[c] = (Real)0;
        df[c] = (Real)0;
    }
    // L: xxx 3ux, xxy uy, xxz uz, xyy ux, xyz 0, xzz ux, yyy 3uy, yyz uz, yzz uy, zzz 3uz
    constexpr int lc[10] = {0, 1, 2, 0, -1, 0, 1, 2, 1, 2};
    constexpr int lm[10] = {3, 1, 1, 1, 0, 1, 3, 1, 1, 3};
    Lk = lc[k] >= 0 ? (Real)lm[k] * u[lc[k]] : (Real)0;
    if (lc[k] >= 0) dL[lc[k]] = (Real)lm[k];
    constexpr int kp[10] = {0, 1, 0, 0, 0, 0, 3, 0, 1, 0};
    kap = (Real)kp[k];
    // f: xxy ux^2, xyy 2 ux uy, xyz ux uz, yyy 3 uy^2, yyz 2 uy uz, yzz uz^2
    fk = (Real)0;
    switch (k) {
        case 1: fk = ux * ux; df[0] = (Real)2 * ux; break;
        case 3: fk = (Real)2 * ux * uy; df[0] = (Real)2 * uy; df[1] = (Real)2 * ux; break;
        case 4: fk = ux * uz; df[0] = uz; df[2] = ux; break;
        case 6: fk = (Real)3 * uy * uy; df[1] = (Real)6 * uy; break;
        case 7: fk = (Real)2 * uy * uz; df[1] = (Real)2 * uz; df[2] = (Real)2 * uy; break;
        case 8: fk = uz * uz; df[2] = (Real)2 * uz; break;
        default: break;
    }
}

template <typename Real, class LAT, bool Z3>
__device__ __forceinline__ void lbm_adjoint_node(const LbmAdjArgs<Real>& a, const int64_t node) {
    constexpr int Q = LAT::Q;
    constexpr double R = lat_r<LAT>();
    const int nx = a.nx, ny = a.ny;
    const int x = (int)(node % nx);
    const int y = Z3 ? (int)((node / nx) % ny) : (int)(node / nx);
    const int z = Z3 ? (int)(node / ((int64_t)nx * ny)) : 0;
    const int64_t nn = a.nnodes;

    // forward intermediates of the node at t
    Real fs[Q];
    if constexpr (Z3)
        pull_node<Real, LAT, true>(a.f, x, y, nx, ny, nn, fs, z, a.nz);
    else
        pull_node<Real, LAT>(a.f, x, y, nx, ny, nn, fs);
    Real rho, jx, jy, jz, pm[6], q3[10];
    node_moments<Real, LAT>(fs, rho, jx, jy, jz, pm, q3);
    const Real gy = a.g_node[node];
    const Real tau = a.tau_node[node];
    const Real om = (Real)1 - (Real)1 / tau, of = (Real)1 - (Real)0.5 / tau;
    const Real inv_rho = (Real)1 / rho;
    const Real ux = jx * inv_rho, uy = (jy + (Real)0.5 * rho * gy) * inv_rho, uz = jz * inv_rho;
    const Real a1y = (Real)-0.5 * rho * gy, rg = rho * gy;
    const Real om1 = (Real)1 - om;

    // adjoints of the combined coefficients from lam_{t+1}(x): f'(+-xi) = w (E +- O)
    const Real* __restrict__ ln = a.lam_next + node;
    Real E0b = (Real)W<LAT>(0) * ln[0];
    Real A1b[3] = {0, 0, 0}, A2b[6] = {0, 0, 0, 0, 0, 0};
    Real B3b[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, t3b[3] = {0, 0, 0};
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int p = opp<LAT>(q);
        if constexpr (q != 0 && q < p) {
            constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
            constexpr double X = R * ex, Y = R * ey, Z = R * ez;
            constexpr double wq = W<LAT>(q);
            const Real lq = ln[(int64_t)q * nn], lp = ln[(int64_t)p * nn];
            const Real evb = (Real)wq * (lq + lp), odb = (Real)wq * (lq - lp);
            E0b += evb;
            if constexpr (ex != 0) A2b[0] += (Real)(0.5 * X * X) * evb;
            if constexpr (ex * ey != 0) A2b[1] += (Real)(X * Y) * evb;
            if constexpr (ex * ez != 0) A2b[2] += (Real)(X * Z) * evb;
            if constexpr (ey != 0) A2b[3] += (Real)(0.5 * Y * Y) * evb;
            if constexpr (ey * ez != 0) A2b[4] += (Real)(Y * Z) * evb;
            if constexpr (ez != 0) A2b[5] += (Real)(0.5 * Z * Z) * evb;
            if constexpr (ex != 0) A1b[0] += (Real)X * odb;
            if constexpr (ey != 0) A1b[1] += (Real)Y * odb;
            if constexpr (ez != 0) A1b[2] += (Real)Z * odb;
            if constexpr (LAT::ORDER >= 3) {
                constexpr double s6 = 1.0 / 6.0;
                if constexpr (ex != 0) {
                    B3b[0] += (Real)(s6 * X * X * X) * odb;
                    t3b[0] -= (Real)(0.5 * X) * odb;
                }
                if constexpr (ex * ey != 0) B3b[1] += (Real)(0.5 * X * X * Y) * odb;
                if constexpr (ex * ez != 0) B3b[2] += (Real)(0.5 * X * X * Z) * odb;
                if constexpr (ex * ey != 0) B3b[3] += (Real)(0.5 * X * Y * Y) * odb;
                if constexpr (ex * ey * ez != 0) B3b[4] += (Real)(X * Y * Z) * odb;
                if constexpr (ex * ez != 0) B3b[5] += (Real)(0.5 * X * Z * Z) * odb;
                if constexpr (ey != 0) {
                    B3b[6] += (Real)(s6 * Y * Y * Y) * odb;
                    t3b[1] -= (Real)(0.5 * Y) * odb;
                }
                if constexpr (ey * ez != 0) B3b[7] += (Real)(0.5 * Y * Y * Z) * odb;
                if constexpr (ey * ez != 0) B3b[8] += (Real)(0.5 * Y * Z * Z) * odb;
                if constexpr (ez != 0) {
                    B3b[9] += (Real)(s6 * Z * Z * Z) * odb;
                    t3b[2] -= (Real)(0.5 * Z) * odb;
                }
            }
        }
    });
    // t3 = trace terms of B3; E0 = A0 - tr(A2) / 2, A0 = rho
    B3b[0] += t3b[0], B3b[3] += t3b[0], B3b[5] += t3b[0];
    B3b[1] += t3b[1], B3b[6] += t3b[1], B3b[8] += t3b[1];
    B3b[2] += t3b[2], B3b[7] += t3b[2], B3b[9] += t3b[2];
    Real rhob = E0b;
    A2b[0] -= (Real)0.5 * E0b, A2b[3] -= (Real)0.5 * E0b, A2b[5] -= (Real)0.5 * E0b;

    // coefficients -> (rho, u, P, Q3, a1y, rg, om, of)
    Real ub[3] = {0, 0, 0}, pb[6], qb[10];
    Real omb = 0, ofb = 0, a1yb = 0, rgb = 0;
    // A1 = (rho ux, rho uy + om a1y + of rg, rho uz)
    rhob += A1b[0] * ux + A1b[1] * uy + A1b[2] * uz;
    ub[0] += A1b[0] * rho, ub[1] += A1b[1] * rho, ub[2] += A1b[2] * rho;
    omb += A1b[1] * a1y, a1yb += A1b[1] * om, ofb += A1b[1] * rg, rgb += A1b[1] * of;
    // A2_ii = rho u_i^2 + om (P_ii - rho (u_i^2 + 1)) [+ 2 of rg uy for yy]
    // A2_ij = rho u_i u_j + om (P_ij - rho u_i u_j) [+ of rg u_other for xy, yz]
    {
        const Real u[3] = {ux, uy, uz};
        constexpr int I[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int i = I[k][0], j = I[k][1];
            const Real b = A2b[k];
            const Real uu = u[i] * u[j];
            const Real diag = i == j ? (Real)1 : (Real)0;
            rhob += b * (uu - om * (uu + diag));
            ub[i] += b * rho * u[j] * om1;
            ub[j] += b * rho * u[i] * om1;
            pb[k] = b * om;
            omb += b * (pm[k] - rho * (uu + diag));
        }
        // force terms: yy 2 of rg uy, xy of rg ux, yz of rg uz
        ub[1] += A2b[3] * (Real)2 * of * rg;
        ofb += A2b[3] * (Real)2 * rg * uy, rgb += A2b[3] * (Real)2 * of * uy;
        ub[0] += A2b[1] * of * rg;
        ofb += A2b[1] * rg * ux, rgb += A2b[1] * of * ux;
        ub[2] += A2b[4] * of * rg;
        ofb += A2b[4] * rg * uz, rgb += A2b[4] * of * uz;
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) qb[k] = (Real)0;
    if constexpr (LAT::ORDER >= 3) {
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            Real M, dM[3], Lk, dL[3], kap, fk, df[3];
            b3_terms<Real>(k, ux, uy, uz, M, dM, Lk, dL, kap, fk, df);
            const Real b = B3b[k];
            rhob += b * (om1 * M - om * Lk);
#pragma unroll
            for (int c = 0; c < 3; ++c) ub[c] += b * (om1 * rho * dM[c] - om * rho * dL[c] + of * rg * df[c]);
            qb[k] = b * om;
            omb += b * (q3[k] - rho * (M + Lk) - kap * a1y);
            a1yb -= b * om * kap;
            ofb += b * rg * fk;
            rgb += b * of * fk;
        }
    }
    // a1y = -rho g / 2, rg = rho g; u = (j + rho g e_y / 2) / rho
    rhob += (Real)-0.5 * gy * a1yb + gy * rgb;
    Real gyb = (Real)-0.5 * rho * a1yb + rho * rgb + (Real)0.5 * ub[1];
    rhob -= (ub[0] * ux + ub[1] * (uy - (Real)0.5 * gy) + ub[2] * uz) * inv_rho;
    const Real jxb = ub[0] * inv_rho, jyb = ub[1] * inv_rho, jzb = ub[2] * inv_rho;
    // om = 1 - 1/tau, of = 1 - 1/(2 tau)
    a.grad_g[node] += gyb;
    a.grad_tau[node] += (omb + (Real)0.5 * ofb) / (tau * tau);

    // mu_q = d rho/dfs_q rhob + ... (the moments are sums over q), then P^T
    constexpr int MV = LAT::MAXV;
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
        constexpr double X = R * ex, Y = R * ey, Z = R * ez;
        Real mu = rhob;
        if constexpr (ex != 0) mu += (Real)X * jxb + (Real)(X * X) * pb[0];
        if constexpr (ey != 0) mu += (Real)Y * jyb + (Real)(Y * Y) * pb[3];
        if constexpr (ez != 0) mu += (Real)Z * jzb + (Real)(Z * Z) * pb[5];
        if constexpr (ex * ey != 0) mu += (Real)(X * Y) * pb[1];
        if constexpr (ex * ez != 0) mu += (Real)(X * Z) * pb[2];
        if constexpr (ey * ez != 0) mu += (Real)(Y * Z) * pb[4];
        if constexpr (LAT::ORDER >= 3) {
            if constexpr (ex != 0) mu += (Real)(X * X * X) * qb[0];
            if constexpr (ex * ey != 0) mu += (Real)(X * X * Y) * qb[1] + (Real)(X * Y * Y) * qb[3];
            if constexpr (ex * ez != 0) mu += (Real)(X * X * Z) * qb[2] + (Real)(X * Z * Z) * qb[5];
            if constexpr (ex * ey * ez != 0) mu += (Real)(X * Y * Z) * qb[4];
            if constexpr (ey != 0) mu += (Real)(Y * Y * Y) * qb[6];
            if constexpr (ey * ez != 0) mu += (Real)(Y * Y * Z) * qb[7] + (Real)(Y * Z * Z) * qb[8];
            if constexpr (ez != 0) mu += (Real)(Z * Z * Z) * qb[9];
        }
        const int sx = x - ex;
        if (sx >= 0 && sx < nx) {
            int64_t srow = wrap_y(y - ey, ny);  // the source row (z - ez) ny + (y - ey)
            if constexpr (Z3) srow += (int64_t)wrap_y(z - ez, a.nz) * ny;
            a.lam[(int64_t)q * nn + srow * nx + sx] = mu;
        } else if constexpr (ex != 0) {
            // a source behind a wall: fs_q = w_q rho_wall(row (y, z))
            const int64_t nrows = Z3 ? (int64_t)ny * a.nz : (int64_t)ny;
            const int64_t row = Z3 ? (int64_t)z * ny + y : (int64_t)y;
            atomicAdd(&a.wall[(sx < 0 ? 0 : nrows) + row], (Real)W<LAT>(q) * mu);
        }
    });
    (void)MV;
}

// The populations leaving through a wall on row (y', z') feed the wall density of row
// (y' + e_y, z' + e_z); their adjoint is that row's wall adjoint times the flux
// normalisation. Task t < 2 nrows: the left (t < nrows) or right wall of source row
// z' ny + y' (z' = 0 for the slab). The wall sums are read from L2.
template <typename Real, class LAT, bool Z3>
__device__ __forceinline__ void adj_wall_row(const LbmAdjArgs<Real>& a, int64_t t) {
    const int ny = a.ny, nx = a.nx;
    const int64_t nrows = Z3 ? (int64_t)ny * a.nz : (int64_t)ny;
    const bool left = t < nrows;
    const int64_t r = left ? t : t - nrows;  // the source row
    const int yr = (int)(r % ny), zr = (int)(r / ny);
    constexpr double inv_flux = 1.0 / wall_flux_norm<LAT>();
    static_for<LAT::Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
        if constexpr (ex != 0) {
            if ((ex < 0) == left) {
                int64_t drow = wrap_y(yr + ey, ny);
                if constexpr (Z3) drow += (int64_t)wrap_y(zr + ez, a.nz) * ny;
                const Real wb = (Real)inv_flux * __ldcg(&a.wall[(left ? 0 : nrows) + drow]);
                Real* lq = a.lam + (int64_t)q * a.nnodes + r * nx;
                if (ex < 0)
                    for (int i = 0; i < -ex; ++i) lq[i] = wb;
                else
                    for (int i = nx - ex; i < nx; ++i) lq[i] = wb;
            }
        }
    });
}

// One thread per node: the collision adjoint and the transposed pull. The last block to
// finish (a ticket after the wall sums of every block) spreads the wall adjoints over the
// populations leaving through the walls, which no node writes, and clears the sums.
template <typename Real, class LAT, bool Z3 = false>
__global__ void __launch_bounds__(128) k_lbm_adj(LbmAdjArgs<Real> a) {
    __shared__ int s_last;
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u < a.nnodes) lbm_adjoint_node<Real, LAT, Z3>(a, u);
    __syncthreads();
    const int64_t nrows = Z3 ? (int64_t)a.ny * a.nz : (int64_t)a.ny;
    unsigned* ticket = reinterpret_cast<unsigned*>(a.wall + 2 * nrows);
    if (threadIdx.x == 0) {
        __threadfence();  // this block's wall sums are visible before its ticket
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int64_t t = threadIdx.x; t < 2 * nrows; t += blockDim.x) adj_wall_row<Real, LAT, Z3>(a, t);
    __syncthreads();
    for (int64_t t = threadIdx.x; t < 2 * nrows; t += blockDim.x) a.wall[t] = (Real)0;
    if (threadIdx.x == 0) *ticket = 0u;
}

// Packed index of the symmetric pair (i, j): xx xy xz yy yz zz.
__device__ __forceinline__ int pidx2(int i, int j) {
    if (i > j) { const int t = i; i = j; j = t; }
    return i == 0 ? j : (i == 1 ? 2 + j : 5);
}
// Coupling-interface loss of the differentiated LBM, one thread per listed node: the Grad
// coefficients of the node's populations (rho, u = j / rho, a2 = P / rho - u u - I,
// a3 = Q3 / rho - sym(u P) / rho + 2 u u u, the comoving coefficients written with the raw
// moments) against 20 targets, summed as squares into *loss, and the adjoint of the
// populations of the node added to lam. Formed in FP64 (a handful of nodes).
template <typename Real, class LAT>
__global__ void k_interface_loss(const Real* __restrict__ f, int64_t nn, const int32_t* __restrict__ nodes,
                                 int n, const Real* __restrict__ targets, double* loss, Real* lam,
                                 unsigned* status) {
    constexpr int Q = LAT::Q;
    constexpr double R = lat_r<LAT>();
    constexpr int I2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    constexpr int I3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                               {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t node = nodes[k];
    if (node < 0 || node >= nn) {
        atomicOr(status, HYB_ST_BAD_INPUT);
        return;
    }
    double rho = 0, J[3] = {0, 0, 0}, P2[6] = {0, 0, 0, 0, 0, 0};
    double P3[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const double xi[3] = {R * E<LAT>(q, 0), R * E<LAT>(q, 1), R * E<LAT>(q, 2)};
        const double fq = (double)f[(int64_t)q * nn + node];
        rho += fq;
#pragma unroll
        for (int i = 0; i < 3; ++i) J[i] += fq * xi[i];
#pragma unroll
        for (int m = 0; m < 6; ++m) P2[m] += fq * xi[I2[m][0]] * xi[I2[m][1]];
#pragma unroll
        for (int m = 0; m < 10; ++m) P3[m] += fq * xi[I3[m][0]] * xi[I3[m][1]] * xi[I3[m][2]];
    });
    const double u[3] = {J[0] / rho, J[1] / rho, J[2] / rho};
    double mb[20], err = 0;
    {
        double mv[20];
        mv[0] = rho;
        for (int i = 0; i < 3; ++i) mv[1 + i] = u[i];
        for (int m = 0; m < 6; ++m) {
            const int i = I2[m][0], j = I2[m][1];
            mv[4 + m] = P2[m] / rho - u[i] * u[j] - (i == j ? 1.0 : 0.0);
        }
        for (int m = 0; m < 10; ++m) {
            const int i = I3[m][0], j = I3[m][1], l = I3[m][2];
            const double S = u[i] * P2[pidx2(j, l)] + u[j] * P2[pidx2(i, l)] + u[l] * P2[pidx2(i, j)];
            mv[10 + m] = P3[m] / rho - S / rho + 2.0 * u[i] * u[j] * u[l];
        }
        for (int m = 0; m < 20; ++m) {
            const double e = mv[m] - (double)targets[20 * (int64_t)k + m];
            err += e * e;
            mb[m] = 2.0 * e;
        }
    }
    atomicAdd(loss, err);
    // reverse: the 20 coefficients -> raw moments
    double rb = mb[0], ub[3] = {mb[1], mb[2], mb[3]}, P2b[6] = {0, 0, 0, 0, 0, 0};
    double P3b[10];
    for (int m = 0; m < 6; ++m) {
        const int i = I2[m][0], j = I2[m][1];
        const double b = mb[4 + m];
        P2b[m] += b / rho;
        rb -= b * P2[m] / (rho * rho);
        ub[i] -= b * u[j];
        ub[j] -= b * u[i];
    }
    for (int m = 0; m < 10; ++m) {
        const int i = I3[m][0], j = I3[m][1], l = I3[m][2];
        const double b = mb[10 + m];
        const int jl = pidx2(j, l), il = pidx2(i, l), ij = pidx2(i, j);
        const double S = u[i] * P2[jl] + u[j] * P2[il] + u[l] * P2[ij];
        P3b[m] = b / rho;
        rb -= b * (P3[m] - S) / (rho * rho);
        ub[i] += b * (-P2[jl] / rho + 2.0 * u[j] * u[l]);
        ub[j] += b * (-P2[il] / rho + 2.0 * u[i] * u[l]);
        ub[l] += b * (-P2[ij] / rho + 2.0 * u[i] * u[j]);
        P2b[jl] -= b * u[i] / rho;
        P2b[il] -= b * u[j] / rho;
        P2b[ij] -= b * u[l] / rho;
    }
    double Jb[3];
    for (int i = 0; i < 3; ++i) {
        Jb[i] = ub[i] / rho;
        rb -= ub[i] * u[i] / rho;
    }
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const double xi[3] = {R * E<LAT>(q, 0), R * E<LAT>(q, 1), R * E<LAT>(q, 2)};
        double g = rb;
        for (int i = 0; i < 3; ++i) g += Jb[i] * xi[i];
        for (int m = 0; m < 6; ++m) g += P2b[m] * xi[I2[m][0]] * xi[I2[m][1]];
        for (int m = 0; m < 10; ++m) g += P3b[m] * xi[I3[m][0]] * xi[I3[m][1]] * xi[I3[m][2]];
        atomicAdd(&lam[(int64_t)q * nn + node], (Real)g);
    });
}

template <typename Real, class LAT>
__global__ void k_lbm_init(Real* f0, Real* f1, int64_t nnodes) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nnodes;
         n += (int64_t)gridDim.x * blockDim.x) {
        static_for<LAT::Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            f0[q * nnodes + n] = (Real)W<LAT>(q);
            f1[q * nnodes + n] = (Real)W<LAT>(q);
        });
    }
}

template <typename Real>
LbmArgs<Real> lbm_args(const Ctx& c, int cur_f) {
    LbmArgs<Real> a;
    a.src = (const Real*)c.st.f[cur_f];
    a.dst = (Real*)c.st.f[cur_f ^ 1];
    a.nx = (int32_t)c.d.nx;
    a.ny = (int32_t)c.d.ny;
    a.nnodes = c.d.nnodes;
    a.om = (Real)(1.0 - 1.0 / c.d.tau);
    a.of = (Real)(1.0 - 0.5 / c.d.tau);
    a.g_step = (Real)c.d.g_step;
    a.g_node = nullptr;
    a.tau_node = (const Real*)c.st.tau_node;  // Kn profile, or null
    a.bgk = c.p.lb_collision;
    a.nz = (int32_t)c.d.nz;
    return a;
}

template <typename Real, class LAT>
cudaError_t lbm_impl(Ctx& c) {
    const LbmArgs<Real> a = lbm_args<Real>(c, c.cur_f);
    const int64_t blocks = (c.d.nnodes + 127) / 128;
    prof_begin(c, K_LBM);
    Launch<LbmArgs<Real>> L{};
    L.one = a;
    L.total = c.d.nnodes;
    const dim3 g((unsigned)blocks), b(128);
    cudaError_t e;
    if (a.nz > 1)  // 3D: periodic in z
        e = a.tau_node ? (a.bgk ? launch_pdl(k_lbm<Real, LAT, false, true, true, true>, g, b, 0, c.stream, L)
                                : launch_pdl(k_lbm<Real, LAT, false, false, true, true>, g, b, 0, c.stream, L))
                       : (a.bgk ? launch_pdl(k_lbm<Real, LAT, false, true, false, true>, g, b, 0, c.stream, L)
                                : launch_pdl(k_lbm<Real, LAT, false, false, false, true>, g, b, 0, c.stream, L));
    else if (a.tau_node)  // Kn profile: per-node tau
        e = a.bgk ? launch_pdl(k_lbm<Real, LAT, false, true, true>, g, b, 0, c.stream, L)
                  : launch_pdl(k_lbm<Real, LAT, false, false, true>, g, b, 0, c.stream, L);
    else
        e = a.bgk ? launch_pdl(k_lbm<Real, LAT, false, true>, g, b, 0, c.stream, L)
                  : launch_pdl(k_lbm<Real, LAT, false>, g, b, 0, c.stream, L);
    prof_end(c, K_LBM);
    return e;
}

template <typename Real, class LAT>
cudaError_t lbm_init_impl(Ctx& c) {
    int64_t g = (c.d.nnodes + 255) / 256;
    if (g > (int64_t)c.num_sms * 16) g = (int64_t)c.num_sms * 16;
    k_lbm_init<Real, LAT><<<(unsigned)g, 256, 0, c.stream>>>((Real*)c.st.f[0], (Real*)c.st.f[1],
                                                             c.d.nnodes);
    c.cur_f = 0;
    return cudaGetLastError();
}


template <typename Real, class LAT>
cudaError_t lbm_nodes_impl(Ctx& c, const void* f_src, void* f_dst, const void* g, const void* tau) {
    LbmArgs<Real> a = lbm_args<Real>(c, c.cur_f);
    a.src = (const Real*)f_src;
    a.dst = (Real*)f_dst;
    a.g_node = (const Real*)g;
    a.tau_node = (const Real*)tau;
    const int64_t blocks = (c.d.nnodes + 127) / 128;
    if (a.nz > 1) {
        if (a.bgk)
            k_lbm_param<Real, LAT, true, true><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
        else
            k_lbm_param<Real, LAT, false, true><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
    } else if (a.bgk) {
        k_lbm_param<Real, LAT, true><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
    } else {
        k_lbm_param<Real, LAT, false><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
    }
    return cudaGetLastError();
}

template <typename Real, class LAT>
cudaError_t lbm_adj_impl(Ctx& c, const void* f, const void* lam_next, void* lam, const void* g,
                         const void* tau, void* grad_g, void* grad_tau, void* wall) {
    LbmAdjArgs<Real> a;
    a.f = (const Real*)f;
    a.lam_next = (const Real*)lam_next;
    a.lam = (Real*)lam;
    a.g_node = (const Real*)g;
    a.tau_node = (const Real*)tau;
    a.grad_g = (Real*)grad_g;
    a.grad_tau = (Real*)grad_tau;
    a.wall = (Real*)wall;
    a.nx = (int32_t)c.d.nx;
    a.ny = (int32_t)c.d.ny;
    a.nz = (int32_t)c.d.nz;
    a.nnodes = c.d.nnodes;
    const int64_t blocks = (c.d.nnodes + 127) / 128;
    if (a.nz > 1)
        k_lbm_adj<Real, LAT, true><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
    else
        k_lbm_adj<Real, LAT><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
    return cudaGetLastError();
}

template <typename Real, class LAT>
cudaError_t loss_impl(Ctx& c, const void* f, const int32_t* nodes, int32_t n, const void* targets,
                      double* loss, void* lam) {
    k_interface_loss<Real, LAT><<<(unsigned)((n + 63) / 64), 64, 0, c.stream>>>(
        (const Real*)f, c.d.nnodes, nodes, n, (const Real*)targets, loss, (Real*)lam,
        (unsigned*)c.st.ctrl + CTRL_STATUS);
    return cudaGetLastError();
}
}  // namespace

size_t lbm_args_bytes(int real_bytes) {
    return real_bytes == 4 ? sizeof(LbmArgs<float>) : sizeof(LbmArgs<double>);
}

void lbm_args_fill(Ctx& c, int cur_f, void* out) {
    if (c.p.real_bytes == 4) {
        const LbmArgs<float> a = lbm_args<float>(c, cur_f);
        std::memcpy(out, &a, sizeof(a));
    } else {
        const LbmArgs<double> a = lbm_args<double>(c, cur_f);
        std::memcpy(out, &a, sizeof(a));
    }
}

namespace {
template <typename Real, class LAT>
cudaError_t batch_lbm_impl(BatchDev& b, int cur_f) {
    Launch<LbmArgs<Real>> L{};
    L.tab = (const LbmArgs<Real>*)b.lbm[cur_f];
    L.pre = b.pre_nodes;
    L.nrep = b.nrep;
    L.total = b.tot_nodes;
    const int64_t blocks = (b.tot_nodes + b.lbm_block - 1) / b.lbm_block;
    if (b.lb_collision)
        return launch_pdl(k_lbm<Real, LAT, true, true>, dim3((unsigned)blocks), dim3(b.lbm_block), 0,
                          b.stream, L);
    return launch_pdl(k_lbm<Real, LAT, true>, dim3((unsigned)blocks), dim3(b.lbm_block), 0, b.stream, L);
}
}  // namespace

cudaError_t launch_batch_lbm(BatchDev& b, int cur_f) {
    if (b.lattice == 39)
        return b.real_bytes == 4 ? batch_lbm_impl<float, D3Q39>(b, cur_f) : batch_lbm_impl<double, D3Q39>(b, cur_f);
    return b.real_bytes == 4 ? batch_lbm_impl<float, D3Q19>(b, cur_f) : batch_lbm_impl<double, D3Q19>(b, cur_f);
}

namespace {

// The LB ghost rows of a streamwise slab (Sec. 3.1: the channel is periodic streamwise; a slab
// holds a range of its rows). side 0 is the slab's lower boundary, side 1 its upper one.
// Pack: the populations a neighbour pulls across that boundary (e_y < 0 at the lower, e_y > 0
// at the upper boundary) from the |e_y| rows of the slab next to it, into buf. Unpack: the
// same populations of the neighbour's rows into the ghost rows (e_y > 0 below the lower
// boundary, e_y < 0 above the upper one). buf holds, for each such q in ascending order, the
// rows at distance k = 0 .. |e_y| - 1 from the boundary, each nz x nx (x fastest).
template <typename Real, class LAT>
__global__ void k_halo(Real* __restrict__ f, Real* __restrict__ buf, int nx, int ny, int nz, int yh,
                       int64_t nn, int side, int unpack) {
    const int64_t plane = (int64_t)nz * nx;
    const bool neg = (side == 0) != (unpack != 0);  // the sign of e_y of the populations in buf
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < plane;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int z = (int)(t / nx), x = (int)(t % nx);
        int64_t off = 0;
        static_for<LAT::Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int ey = E<LAT>(q, 1);
            const int e = neg ? -ey : ey;
            for (int k = 0; k < e; ++k) {
                const int y = unpack ? (side == 0 ? yh - 1 - k : ny - yh + k)
                                     : (side == 0 ? yh + k : ny - yh - 1 - k);
                const int64_t node = ((int64_t)z * ny + y) * nx + x;
                const int64_t bi = off + (int64_t)k * plane + t;
                if (unpack)
                    f[(int64_t)q * nn + node] = buf[bi];
                else
                    buf[bi] = f[(int64_t)q * nn + node];
            }
            if (e > 0) off += (int64_t)e * plane;
        });
    }
}

// Values per side: sum over q of max(e_y, 0), times nz nx.
template <class LAT>
int64_t halo_rows() {
    int64_t s = 0;
    for (int q = 0; q < LAT::Q; ++q) s += LatTab<LAT>::e(q, 1) > 0 ? LatTab<LAT>::e(q, 1) : 0;
    return s;
}

template <typename Real, class LAT>
cudaError_t halo_impl(Ctx& c, int side, void* buf, int unpack) {
    const int64_t plane = c.d.nz * c.d.nx;
    int64_t g = (plane + 255) / 256;
    if (g > (int64_t)c.num_sms * 8) g = (int64_t)c.num_sms * 8;
    k_halo<Real, LAT><<<(unsigned)g, 256, 0, c.stream>>>((Real*)c.st.f[c.cur_f], (Real*)buf,
                                                          (int)c.d.nx, (int)c.d.ny, (int)c.d.nz,
                                                          (int)c.d.yh, c.d.nnodes, side, unpack);
    return cudaGetLastError();
}

}  // namespace

int64_t lbm_halo_values(const Ctx& c) {
    return (c.p.lattice == 39 ? halo_rows<D3Q39>() : halo_rows<D3Q19>()) * c.d.nz * c.d.nx;
}

cudaError_t launch_lbm_halo(Ctx& c, int side, void* buf, int unpack) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? halo_impl<float, D3Q39>(c, side, buf, unpack)
                                   : halo_impl<double, D3Q39>(c, side, buf, unpack);
    return c.p.real_bytes == 4 ? halo_impl<float, D3Q19>(c, side, buf, unpack)
                               : halo_impl<double, D3Q19>(c, side, buf, unpack);
}

cudaError_t launch_lbm_step(Ctx& c) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? lbm_impl<float, D3Q39>(c) : lbm_impl<double, D3Q39>(c);
    return c.p.real_bytes == 4 ? lbm_impl<float, D3Q19>(c) : lbm_impl<double, D3Q19>(c);
}

cudaError_t launch_lbm_init(Ctx& c) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? lbm_init_impl<float, D3Q39>(c) : lbm_init_impl<double, D3Q39>(c);
    return c.p.real_bytes == 4 ? lbm_init_impl<float, D3Q19>(c) : lbm_init_impl<double, D3Q19>(c);
}


cudaError_t launch_lbm_step_nodes(Ctx& c, const void* f_src, void* f_dst, const void* g, const void* tau) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? lbm_nodes_impl<float, D3Q39>(c, f_src, f_dst, g, tau)
                                   : lbm_nodes_impl<double, D3Q39>(c, f_src, f_dst, g, tau);
    return c.p.real_bytes == 4 ? lbm_nodes_impl<float, D3Q19>(c, f_src, f_dst, g, tau)
                               : lbm_nodes_impl<double, D3Q19>(c, f_src, f_dst, g, tau);
}

cudaError_t launch_lbm_adjoint_step(Ctx& c, const void* f, const void* lam_next, void* lam,
                                    const void* g, const void* tau, void* grad_g, void* grad_tau,
                                    void* wall) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4
                   ? lbm_adj_impl<float, D3Q39>(c, f, lam_next, lam, g, tau, grad_g, grad_tau, wall)
                   : lbm_adj_impl<double, D3Q39>(c, f, lam_next, lam, g, tau, grad_g, grad_tau, wall);
    return c.p.real_bytes == 4
               ? lbm_adj_impl<float, D3Q19>(c, f, lam_next, lam, g, tau, grad_g, grad_tau, wall)
               : lbm_adj_impl<double, D3Q19>(c, f, lam_next, lam, g, tau, grad_g, grad_tau, wall);
}

cudaError_t launch_interface_loss(Ctx& c, const void* f, const int32_t* nodes, int32_t n,
                                  const void* targets, double* loss, void* lam) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? loss_impl<float, D3Q39>(c, f, nodes, n, targets, loss, lam)
                                   : loss_impl<double, D3Q39>(c, f, nodes, n, targets, loss, lam);
    return c.p.real_bytes == 4 ? loss_impl<float, D3Q19>(c, f, nodes, n, targets, loss, lam)
                               : loss_impl<double, D3Q19>(c, f, nodes, n, targets, loss, lam);
}

}  // namespace hyb
