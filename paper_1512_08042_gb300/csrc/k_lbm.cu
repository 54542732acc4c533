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
//   f_eq = w rho [1 + xi.u + ((xi.u)^2 - u^2)/2 + (xi.u)((xi.u)^2 - 3u^2)/6],
//   non-equilibrium Hermite coefficients a1 = -rho g / 2, a2 = Pi - rho(uu + I),
//   a3 = Qm - rho(uuu + sym(u I)) - sym(a1 I),
//   f' = f_eq + (1 - 1/tau) w [a1.xi + a2:H2/2 + a3:H3/6] + (1 - 1/(2 tau)) F,
//   F = w rho [g.xi + (g.xi)(u.xi) - g.u + ((g.xi)(u.xi)^2 - (g.xi)u^2 - 2(u.xi)(g.u))/2].
// Every lattice constant is a compile-time value, so terms with zero speed components
// vanish at compile time.
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

__device__ __forceinline__ int wrap_y(int v, int ny) {
    while (v < 0) v += ny;
    while (v >= ny) v -= ny;
    return v;
}

template <typename Real, class LAT>
__global__ void __launch_bounds__(128) k_lbm(LbmArgs<Real> a) {
    constexpr int Q = LAT::Q;
    constexpr double R = lat_r<LAT>();
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= a.nnodes) return;
    const int nx = a.nx, ny = a.ny;
    const int x = (int)(node % nx), y = (int)(node / nx);
    const int64_t nn = a.nnodes;
    const Real* __restrict__ src = a.src;

    // Wall densities for nodes whose pull reaches through a wall: the mass leaving through
    // the wall on this row, re-emitted by the wall Maxwellian at rest.
    Real rhoL = (Real)0, rhoR = (Real)0;
    if (x < LAT::MAXV || x >= nx - LAT::MAXV) {
        Real ml = (Real)0, mr = (Real)0;
        static_for<Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1);
            if constexpr (ex < 0) {
                const int sy = wrap_y(y - ey, ny);
#pragma unroll
                for (int i = 0; i < -ex; ++i) ml += src[q * nn + (int64_t)sy * nx + i];
            }
            if constexpr (ex > 0) {
                const int sy = wrap_y(y - ey, ny);
#pragma unroll
                for (int i = 0; i < ex; ++i) mr += src[q * nn + (int64_t)sy * nx + (nx - ex + i)];
            }
        });
        constexpr double inv_flux = 1.0 / wall_flux_norm<LAT>();
        rhoL = ml * (Real)inv_flux;
        rhoR = mr * (Real)inv_flux;
    }

    Real fs[Q];
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1);
        const int sx = x - ex;
        const int sy = (ey == 0) ? y : wrap_y(y - ey, ny);
        if (sx < 0)
            fs[q] = (Real)W<LAT>(q) * rhoL;
        else if (sx >= nx)
            fs[q] = (Real)W<LAT>(q) * rhoR;
        else
            fs[q] = src[q * nn + (int64_t)sy * nx + sx];
    });

    // moments
    Real rho = 0, jx = 0, jy = 0, jz = 0;
    Real pxx = 0, pxy = 0, pxz = 0, pyy = 0, pyz = 0, pzz = 0;
    Real q3[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
        const Real f = fs[q];
        rho += f;
        if constexpr (ex != 0) jx += f * (Real)(R * ex);
        if constexpr (ey != 0) jy += f * (Real)(R * ey);
        if constexpr (ez != 0) jz += f * (Real)(R * ez);
        if constexpr (ex != 0) pxx += f * (Real)(R * R * ex * ex);
        if constexpr (ex * ey != 0) pxy += f * (Real)(R * R * ex * ey);
        if constexpr (ex * ez != 0) pxz += f * (Real)(R * R * ex * ez);
        if constexpr (ey != 0) pyy += f * (Real)(R * R * ey * ey);
        if constexpr (ey * ez != 0) pyz += f * (Real)(R * R * ey * ez);
        if constexpr (ez != 0) pzz += f * (Real)(R * R * ez * ez);
        if constexpr (LAT::ORDER >= 3) {
            constexpr double R3 = R * R * R;
            if constexpr (ex != 0) q3[0] += f * (Real)(R3 * ex * ex * ex);
            if constexpr (ex * ey != 0) q3[1] += f * (Real)(R3 * ex * ex * ey);
            if constexpr (ex * ez != 0) q3[2] += f * (Real)(R3 * ex * ex * ez);
            if constexpr (ex * ey != 0) q3[3] += f * (Real)(R3 * ex * ey * ey);
            if constexpr (ex * ey * ez != 0) q3[4] += f * (Real)(R3 * ex * ey * ez);
            if constexpr (ex * ez != 0) q3[5] += f * (Real)(R3 * ex * ez * ez);
            if constexpr (ey != 0) q3[6] += f * (Real)(R3 * ey * ey * ey);
            if constexpr (ey * ez != 0) q3[7] += f * (Real)(R3 * ey * ey * ez);
            if constexpr (ey * ez != 0) q3[8] += f * (Real)(R3 * ey * ez * ez);
            if constexpr (ez != 0) q3[9] += f * (Real)(R3 * ez * ez * ez);
        }
    });

    const Real gy = a.g_step;
    const Real inv_rho = (Real)1 / rho;
    const Real ux = jx * inv_rho, uy = (jy + (Real)0.5 * rho * gy) * inv_rho, uz = jz * inv_rho;
    const Real u2 = ux * ux + uy * uy + uz * uz;
    const Real a1y = (Real)-0.5 * rho * gy;  // H1 part of f_neq
    // a2 = Pi - rho (uu + I)
    const Real bxx = pxx - rho * (ux * ux + (Real)1), byy = pyy - rho * (uy * uy + (Real)1),
               bzz = pzz - rho * (uz * uz + (Real)1);
    const Real bxy = pxy - rho * ux * uy, bxz = pxz - rho * ux * uz, byz = pyz - rho * uy * uz;
    const Real tr2 = bxx + byy + bzz;
    // a3 = Qm - rho(uuu + sym(u I)) - sym(a1 I); a1 has only a y component
    Real c3[10];
    Real t3x = 0, t3y = 0, t3z = 0;
    if constexpr (LAT::ORDER >= 3) {
        c3[0] = q3[0] - rho * (ux * ux * ux + (Real)3 * ux);
        c3[1] = q3[1] - rho * (ux * ux * uy + uy) - a1y;
        c3[2] = q3[2] - rho * (ux * ux * uz + uz);
        c3[3] = q3[3] - rho * (ux * uy * uy + ux);
        c3[4] = q3[4] - rho * (ux * uy * uz);
        c3[5] = q3[5] - rho * (ux * uz * uz + ux);
        c3[6] = q3[6] - rho * (uy * uy * uy + (Real)3 * uy) - (Real)3 * a1y;
        c3[7] = q3[7] - rho * (uy * uy * uz + uz);
        c3[8] = q3[8] - rho * (uy * uz * uz + uy) - a1y;
        c3[9] = q3[9] - rho * (uz * uz * uz + (Real)3 * uz);
        t3x = c3[0] + c3[3] + c3[5];
        t3y = c3[1] + c3[6] + c3[8];
        t3z = c3[2] + c3[7] + c3[9];
    }
    const Real om = a.om;
    const Real of = a.of;
    const Real gu = gy * uy;
    Real* __restrict__ dst = a.dst;

    static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int ex = E<LAT>(q, 0), ey = E<LAT>(q, 1), ez = E<LAT>(q, 2);
        constexpr double X = R * ex, Y = R * ey, Z = R * ez;
        Real xu = (Real)0;
        if constexpr (ex != 0) xu += (Real)X * ux;
        if constexpr (ey != 0) xu += (Real)Y * uy;
        if constexpr (ez != 0) xu += (Real)Z * uz;
        Real feq = (Real)1 + xu + (Real)0.5 * (xu * xu - u2);
        if constexpr (LAT::ORDER >= 3) feq += (Real)(1.0 / 6.0) * xu * (xu * xu - (Real)3 * u2);
        // regularised non-equilibrium part
        Real h2 = -tr2;
        if constexpr (ex != 0) h2 += (Real)(X * X) * bxx;
        if constexpr (ey != 0) h2 += (Real)(Y * Y) * byy;
        if constexpr (ez != 0) h2 += (Real)(Z * Z) * bzz;
        if constexpr (ex * ey != 0) h2 += (Real)(2 * X * Y) * bxy;
        if constexpr (ex * ez != 0) h2 += (Real)(2 * X * Z) * bxz;
        if constexpr (ey * ez != 0) h2 += (Real)(2 * Y * Z) * byz;
        Real neq = (Real)0.5 * h2;
        if constexpr (ey != 0) neq += (Real)Y * a1y;
        if constexpr (LAT::ORDER >= 3) {
            Real h3 = (Real)0;
            if constexpr (ex != 0) h3 += (Real)(X * X * X) * c3[0] - (Real)(3 * X) * t3x;
            if constexpr (ex * ey != 0) h3 += (Real)(3 * X * X * Y) * c3[1];
            if constexpr (ex * ez != 0) h3 += (Real)(3 * X * X * Z) * c3[2];
            if constexpr (ex * ey != 0) h3 += (Real)(3 * X * Y * Y) * c3[3];
            if constexpr (ex * ey * ez != 0) h3 += (Real)(6 * X * Y * Z) * c3[4];
            if constexpr (ex * ez != 0) h3 += (Real)(3 * X * Z * Z) * c3[5];
            if constexpr (ey != 0) h3 += (Real)(Y * Y * Y) * c3[6] - (Real)(3 * Y) * t3y;
            if constexpr (ey * ez != 0) h3 += (Real)(3 * Y * Y * Z) * c3[7];
            if constexpr (ey * ez != 0) h3 += (Real)(3 * Y * Z * Z) * c3[8];
            if constexpr (ez != 0) h3 += (Real)(Z * Z * Z) * c3[9] - (Real)(3 * Z) * t3z;
            neq += (Real)(1.0 / 6.0) * h3;
        }
        // Hermite force term, g along y
        const Real gx = (ey != 0) ? (Real)Y * gy : (Real)0;  // g . xi
        Real F = gx + gx * xu - gu;
        if constexpr (LAT::ORDER >= 3)
            F += (Real)0.5 * (gx * xu * xu - gx * u2 - (Real)2 * xu * gu);
        const Real out = (Real)W<LAT>(q) * (rho * feq + om * neq + of * rho * F);
        dst[q * nn + node] = out;
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

template <typename Real, class LAT>
cudaError_t lbm_impl(Ctx& c) {
    LbmArgs<Real> a;
    a.src = (const Real*)c.st.f[c.cur_f];
    a.dst = (Real*)c.st.f[c.cur_f ^ 1];
    a.nx = (int32_t)c.d.nx;
    a.ny = (int32_t)c.d.ny;
    a.nnodes = c.d.nnodes;
    a.om = (Real)(1.0 - 1.0 / c.d.tau);
    a.of = (Real)(1.0 - 0.5 / c.d.tau);
    a.g_step = (Real)c.d.g_step;
    const int64_t blocks = (c.d.nnodes + 127) / 128;
    prof_begin(c, K_LBM);
    k_lbm<Real, LAT><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
    prof_end(c, K_LBM);
    return cudaGetLastError();
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
