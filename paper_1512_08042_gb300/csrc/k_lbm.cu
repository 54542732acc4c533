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

// One node of one context.
template <typename Real, class LAT>
__device__ __forceinline__ void lbm_node(const LbmArgs<Real>& a, const int64_t node) {
    constexpr int Q = LAT::Q;
    constexpr double R = lat_r<LAT>();
    const int nx = a.nx, ny = a.ny;
    const int x = (int)(node % nx), y = (int)(node / nx);
    const int64_t nn = a.nnodes;
    const Real* __restrict__ src = a.src;

    // Row offsets y' * nx of the pull sources y' = y - ey (periodic), ey = -MAXV..MAXV.
    constexpr int MV = LAT::MAXV;
    int rowoff[2 * MV + 1];
#pragma unroll
    for (int i = 0; i < 2 * MV + 1; ++i) rowoff[i] = wrap_y(y - (i - MV), ny) * nx;

    // Wall densities for nodes whose pull reaches through a wall: the mass leaving through
    // the wall on this row, re-emitted by the wall Maxwellian at rest.
    Real rhoL = (Real)0, rhoR = (Real)0;
    if (x < MV || x >= nx - MV) {
        Real ml = (Real)0, mr = (Real)0;
        static_for<Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1);
            const Real* __restrict__ sq = src + (int64_t)q * nn + rowoff[ey + MV];
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

    // pull streaming; sources behind a wall take the wall Maxwellian
    Real fs[Q];
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1);
        const Real* __restrict__ sq = src + (int64_t)q * nn;
        const int sx = x - ex;
        const int off = rowoff[ey + MV] + sx;
        if constexpr (ex > 0)
            fs[q] = sx < 0 ? (Real)W<LAT>(q) * rhoL : sq[off];
        else if constexpr (ex < 0)
            fs[q] = sx >= nx ? (Real)W<LAT>(q) * rhoR : sq[off];
        else
            fs[q] = sq[off];
    });

    // moments, from the pair sums s and differences d
    Real rho = fs[0], jx = 0, jy = 0, jz = 0;
    Real pxx = 0, pxy = 0, pxz = 0, pyy = 0, pyz = 0, pzz = 0;
    Real q3[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
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
            if constexpr (ex != 0) pxx += sm * (Real)(R * R * ex * ex);
            if constexpr (ex * ey != 0) pxy += sm * (Real)(R * R * ex * ey);
            if constexpr (ex * ez != 0) pxz += sm * (Real)(R * R * ex * ez);
            if constexpr (ey != 0) pyy += sm * (Real)(R * R * ey * ey);
            if constexpr (ey * ez != 0) pyz += sm * (Real)(R * R * ey * ez);
            if constexpr (ez != 0) pzz += sm * (Real)(R * R * ez * ez);
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

    const Real gy = a.g_step;
    const Real om = a.om;
    const Real of = a.of;
    const Real inv_rho = (Real)1 / rho;
    const Real ux = jx * inv_rho, uy = (jy + (Real)0.5 * rho * gy) * inv_rho, uz = jz * inv_rho;
    const Real a1y = (Real)-0.5 * rho * gy;  // H1 part of f_neq
    const Real rg = rho * gy;
    // combined coefficients of the post-collision series
    const Real A0 = rho;
    const Real A1x = rho * ux, A1y = rho * uy + om * a1y + of * rg, A1z = rho * uz;
    // a2 = Pi - rho (uu + I); A2 = rho uu + om a2 + of rho (gu + ug)
    const Real Axx = rho * ux * ux + om * (pxx - rho * (ux * ux + (Real)1));
    const Real Ayy = rho * uy * uy + om * (pyy - rho * (uy * uy + (Real)1)) + of * (Real)2 * rg * uy;
    const Real Azz = rho * uz * uz + om * (pzz - rho * (uz * uz + (Real)1));
    const Real Axy = rho * ux * uy + om * (pxy - rho * ux * uy) + of * rg * ux;
    const Real Axz = rho * ux * uz + om * (pxz - rho * ux * uz);
    const Real Ayz = rho * uy * uz + om * (pyz - rho * uy * uz) + of * rg * uz;
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
        B3[0] = rho * ux * ux * ux + om * c0;
        B3[1] = rho * ux * ux * uy + om * c1 + of * rg * ux * ux;
        B3[2] = rho * ux * ux * uz + om * c2;
        B3[3] = rho * ux * uy * uy + om * c3 + of * (Real)2 * rg * ux * uy;
        B3[4] = rho * ux * uy * uz + om * c4 + of * rg * ux * uz;
        B3[5] = rho * ux * uz * uz + om * c5;
        B3[6] = rho * uy * uy * uy + om * c6 + of * (Real)3 * rg * uy * uy;
        B3[7] = rho * uy * uy * uz + om * c7 + of * (Real)2 * rg * uy * uz;
        B3[8] = rho * uy * uz * uz + om * c8 + of * rg * uz * uz;
        B3[9] = rho * uz * uz * uz + om * c9;
        t3x = B3[0] + B3[3] + B3[5];
        t3y = B3[1] + B3[6] + B3[8];
        t3z = B3[2] + B3[7] + B3[9];
    }
    Real* __restrict__ dst = a.dst + node;

    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int p = opp<LAT>(q);
        if constexpr (q == 0) {
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
            dst[(int64_t)q * nn] = (Real)wq * (ev + od);
            dst[(int64_t)p * nn] = (Real)wq * (ev - od);
        }
    });
}

// One thread per node (the nodes of all replicas in the batch form).
template <typename Real, class LAT, bool BATCH>
__global__ void __launch_bounds__(128) k_lbm(Launch<LbmArgs<Real>> L) {
    pdl_begin();
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= L.total) return;
    if constexpr (BATCH) {
        const int r = replica_of(L.pre, L.nrep, u);
        lbm_node<Real, LAT>(L.tab[r], u - L.pre[r]);
    } else {
        lbm_node<Real, LAT>(L.one, u);
    }
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
    const cudaError_t e = launch_pdl(k_lbm<Real, LAT, false>, dim3((unsigned)blocks), dim3(128), 0, c.stream, L);
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
    return launch_pdl(k_lbm<Real, LAT, true>, dim3((unsigned)blocks), dim3(b.lbm_block), 0, b.stream, L);
}
}  // namespace

cudaError_t launch_batch_lbm(BatchDev& b, int cur_f) {
    if (b.lattice == 39)
        return b.real_bytes == 4 ? batch_lbm_impl<float, D3Q39>(b, cur_f) : batch_lbm_impl<double, D3Q39>(b, cur_f);
    return b.real_bytes == 4 ? batch_lbm_impl<float, D3Q19>(b, cur_f) : batch_lbm_impl<double, D3Q19>(b, cur_f);
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

}  // namespace hyb
