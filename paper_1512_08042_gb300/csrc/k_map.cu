// The two kinetic mappings of Sec. 2. The Grad/Hermite coefficients are formed in FP64;
// populations and particle state are Real (float or double).
//
// k_d2l (DSMC2LB, Sec. 2.1): one warp per coupling node. The cumulative sums of the
// node's DSMC cell give rho = <N>/ppc, the per-particle raw moments <v>, <vv>, <vvv> (one
// FP64 reciprocal of the count) and the raw Hermite coefficients a0 = rho, a1 = rho <v>,
// a2 = rho(<vv> - I), a3 = rho(<vvv> - sym(<v> I)), all in FP64 (the stress and heat-flux
// parts are differences of nearly equal moments); the populations
// f_a = w_a sum_{n<=N} a^(n):H^(n)(xi_a)/n! (Eq. discretefunctions) are evaluated in the
// state precision from the coefficients rounded to it.
//
// LB2DSMC (Sec. 2.2, Table 1), k_l2d: one block per coupling cell. Warp 0 forms, in FP64, the
// mean populations of the cell's lb_ratio^2 nodes, rho and u, the comoving coefficients
// a2 = sum f c c / rho - I and a3 = sum f c c c / rho (c = xi - u), M, C = 1 + 30 M (Eq. C)
// and the particle count floor(rho ppc + U); the other warps wait (trials drawn meanwhile
// took issue slots from warp 0 and lengthened the path). The cell's trial stream is then
// evaluated 256 trials at a time in the state precision, with the coefficients rounded to
// it: Box-Muller xi from the unit Maxwellian, accepted when C R <= G(xi),
// G = 1 + a2:H2/2 + a3:H3/6 (Eq. distr_outeq); the k-th accepted trial becomes the k-th
// particle of the cell's bin (replacing the old ones), velocity xi + u (Eq. step6 in c_th
// units), position uniform in the cell from the same trial's draws.
// Draws are keyed by (cell, step, purpose, trial index), so the results do not depend on
// the launch shape.
#include <cstring>
#include <mutex>

#include "dsmc_move.cuh"

// Fixed scratch of map_lbm_to_dsmc_noalloc: one Grad record per coupling cell, for callers
// that cannot hand the library any device memory beyond the state itself. The array lives
// in every device that loads the library until the process exits. Host code must not pass
// `g_l2d_scratch` itself to a kernel (on the host it names a stand-in, not device memory):
// its device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) hyb::GradRec g_l2d_scratch[HYB_NOALLOC_MAX_CELLS];

namespace hyb {

namespace {

// Lattice speeds xi = r e in the state precision (r e formed in double and rounded, as the
// oracle does) and weights, as device tables built at compile time, for lanes that each
// handle a different population.
template <class LAT, typename Real>
struct LatXi {
    Real x[3 * LAT::Q];
    Real w[LAT::Q];
};
template <class LAT, typename Real>
constexpr LatXi<LAT, Real> make_xi() {
    LatXi<LAT, Real> t{};
    for (int a = 0; a < LAT::Q; ++a) {
        for (int i = 0; i < 3; ++i) t.x[3 * a + i] = (Real)(lat_r<LAT>() * (double)LatTab<LAT>::e(a, i));
        t.w[a] = (Real)LatTab<LAT>::w(a);
    }
    return t;
}
__device__ const LatXi<D3Q39, float> g_xi39f = make_xi<D3Q39, float>();
__device__ const LatXi<D3Q39, double> g_xi39d = make_xi<D3Q39, double>();
__device__ const LatXi<D3Q19, float> g_xi19f = make_xi<D3Q19, float>();
__device__ const LatXi<D3Q19, double> g_xi19d = make_xi<D3Q19, double>();

template <class LAT, typename Real>
__device__ __forceinline__ const LatXi<LAT, Real>& lat_xi() {
    if constexpr (LAT::Q == 39) {
        if constexpr (sizeof(Real) == 4)
            return g_xi39f;
        else
            return g_xi39d;
    } else {
        if constexpr (sizeof(Real) == 4)
            return g_xi19f;
        else
            return g_xi19d;
    }
}

// DSMC2LB: one warp per coupling node. Lanes 0-19 read the cell's 20 sums and scale them
// by one FP64 reciprocal of the particle count; the coefficients (one per lane, state
// precision) are broadcast and each lane evaluates one or two populations.
template <typename Real, class LAT>
__device__ __forceinline__ void d2l_entries(const MapArgs<Real>& a, int first, int stride) {
    const LatXi<LAT, Real>& lt = lat_xi<LAT, Real>();
    const Real* sx = lt.x;
    const Real* sw = lt.w;
    const unsigned lane = lane_id();
    const uint32_t S = a.ctrl[CTRL_NSAMPLES];
    for (int t = first; t < a.n; t += stride) {
        const int32_t node = a.list[t];
        if (node < 0 || (int64_t)node >= a.nnodes) {
            if (lane == 0) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            continue;
        }
        // node (z ny + y) nx + x lies in cell (iz ncy + iy) ncx + ix (z = 0 in 2D); a slab's
        // ghost rows (the yh rows below and above its own) belong to no cell of the context
        const int x = node % a.nx, y = (node / a.nx) % a.ny - a.yh, z = node / (a.nx * a.ny);
        if (y < 0 || y >= a.ncy * a.lb_ratio) {
            if (lane == 0) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            continue;
        }
        const int64_t cell =
            ((int64_t)(z / a.lb_ratio) * a.ncy + y / a.lb_ratio) * a.ncx + (x / a.lb_ratio);
        const double* m = a.acc + cell * kMoments;
        const double mk = lane < (unsigned)kMoments ? m[lane] : 0.0;
        const double NS = __shfl_sync(kFull, mk, 0);
        if (S == 0 || !(NS > 0.0)) {
            if (lane == 0) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            continue;
        }
        // per-particle moments, lane k: <v> (1-3), <vv> (4-9), <vvv> (10-19), and the raw
        // Hermite coefficients, in FP64; the reciprocal of the count is formed by one lane
        double inv = 0.0;
        if (lane == 0) inv = 1.0 / NS;
        inv = __shfl_sync(kFull, inv, 0);
        const double mr = mk * inv;
        const double rho = NS / ((double)S * (double)a.ppc);
        const double m1x = __shfl_sync(kFull, mr, 1);
        const double m1y = __shfl_sync(kFull, mr, 2);
        const double m1z = __shfl_sync(kFull, mr, 3);
        double sub = 0.0;
        switch (lane) {
            case 4: case 7: case 9: sub = 1.0; break;       // xx yy zz
            case 10: sub = 3.0 * m1x; break;                // xxx
            case 11: sub = m1y; break;                      // xxy
            case 12: sub = m1z; break;                      // xxz
            case 13: sub = m1x; break;                      // xyy
            case 15: sub = m1x; break;                      // xzz
            case 16: sub = 3.0 * m1y; break;                // yyy
            case 17: sub = m1z; break;                      // yyz
            case 18: sub = m1y; break;                      // yzz
            case 19: sub = 3.0 * m1z; break;                // zzz
            default: break;
        }
        double coef = lane == 0 ? rho : rho * (mr - sub);
        if (a.eq_mode && lane >= 4u && lane < (unsigned)kMoments) {
            // the local equilibrium of rho and u (Sec. 4, Eq. feq_dsmc): a2 = rho u u,
            // a3 = rho u u u
            constexpr int I[16][3] = {{0, 0, -1}, {0, 1, -1}, {0, 2, -1}, {1, 1, -1}, {1, 2, -1},
                                      {2, 2, -1}, {0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1},
                                      {0, 1, 2}, {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2},
                                      {2, 2, 2}};
            const double uu[3] = {m1x, m1y, m1z};
            const int* ix = I[lane - 4u];
            coef = rho * uu[ix[0]] * uu[ix[1]];
            if (ix[2] >= 0) coef = coef * uu[ix[2]];
        }
        const Real coef_r = (Real)coef;
        Real cf[kMoments];
#pragma unroll
        for (int k = 0; k < kMoments; ++k) cf[k] = __shfl_sync(kFull, coef_r, k);
        const Real* a2 = cf + 4;
        const Real* a3 = cf + 10;
        const Real tx = a3[0] + a3[3] + a3[5], ty = a3[1] + a3[6] + a3[8], tz = a3[2] + a3[7] + a3[9];
        const Real tr2 = a2[0] + a2[3] + a2[5];
#pragma unroll
        for (int h = 0; h < (LAT::Q + 31) / 32; ++h) {
            const int q = (int)lane + 32 * h;
            if (q < LAT::Q) {
                const Real X = sx[3 * q], Y = sx[3 * q + 1], Z = sx[3 * q + 2];
                const Real h2 = a2[0] * X * X + a2[3] * Y * Y + a2[5] * Z * Z - tr2 +
                                (Real)2 * (a2[1] * X * Y + a2[2] * X * Z + a2[4] * Y * Z);
                Real sum = cf[0] + cf[1] * X + cf[2] * Y + cf[3] * Z + (Real)0.5 * h2;
                if (LAT::ORDER >= 3) {
                    const Real cubic = a3[0] * X * X * X + (Real)3 * a3[1] * X * X * Y +
                                       (Real)3 * a3[2] * X * X * Z + (Real)3 * a3[3] * X * Y * Y +
                                       (Real)6 * a3[4] * X * Y * Z + (Real)3 * a3[5] * X * Z * Z +
                                       a3[6] * Y * Y * Y + (Real)3 * a3[7] * Y * Y * Z +
                                       (Real)3 * a3[8] * Y * Z * Z + a3[9] * Z * Z * Z;
                    sum += (cubic - (Real)3 * (tx * X + ty * Y + tz * Z)) * (Real)(1.0 / 6.0);
                }
                a.f[(int64_t)q * a.nnodes + node] = sw[q] * sum;
            }
        }
    }
}

// DSMC2LB: one warp per listed node (the listed nodes of all replicas in the batch form).
template <typename Real, class LAT, bool BATCH>
__global__ void __launch_bounds__(256) k_d2l(Launch<MapArgs<Real>> L) {
    pdl_begin();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if constexpr (BATCH) {
        if (gw >= L.total) return;
        const int r = replica_of(L.pre, L.nrep, gw);
        const MapArgs<Real>& a = L.tab[r];
        d2l_entries<Real, LAT>(a, (int)(gw - L.pre[r]), a.n);
    } else {
        d2l_entries<Real, LAT>(L.one, (int)gw, (int)(((int64_t)gridDim.x * blockDim.x) >> 5));
    }
}

// Sums each of the N values (N a power of two, at most 32) over the 32 lanes, combining
// lanes l and l ^ o for o = 16, 8, 4, 2, 1 in turn; while N > 1 each lane keeps half of its
// values at every step (a halving exchange). Lane l ends with the total of value
// l >> (5 - log2 N) in v[0]. Every total is formed by the same tree of additions as a
// butterfly over each value alone: the pairwise order of the oracle after its first level.
template <typename Real, int N>
__device__ __forceinline__ void halving_sum(Real (&v)[N], unsigned lane) {
    int o = 16;
#pragma unroll
    for (int len = N / 2; len >= 1; len >>= 1, o >>= 1) {
        const bool hi = (lane & (unsigned)o) != 0;
#pragma unroll
        for (int q = 0; q < len; ++q) {
            const Real send = hi ? v[q] : v[q + len];
            const Real keep = hi ? v[q + len] : v[q];
            v[q] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
#pragma unroll
    for (; o >= 1; o >>= 1) v[0] = v[0] + __shfl_xor_sync(kFull, v[0], o);
}

// G of Eq. distr_outeq in the state precision, from the comoving coefficients packed by
// symmetry, with the grouping of the Table 1 sums fixed (distinct entries times their
// multiplicity) so that the accept decision is reproducible.
template <typename Real, int ORDER>
__device__ __forceinline__ Real grad_G(const Real* a2, const Real* a3, Real X, Real Y, Real Z) {
    const Real h2 = a2[0] * (X * X - (Real)1) + a2[3] * (Y * Y - (Real)1) +
                    a2[5] * (Z * Z - (Real)1) +
                    (Real)2 * (a2[1] * X * Y + a2[2] * X * Z + a2[4] * Y * Z);
    Real G = (Real)1 + (Real)0.5 * h2;
    if (ORDER >= 3) {
        const Real cubic = a3[0] * X * X * X + (Real)3 * a3[1] * X * X * Y +
                           (Real)3 * a3[2] * X * X * Z + (Real)3 * a3[3] * X * Y * Y +
                           (Real)6 * a3[4] * X * Y * Z + (Real)3 * a3[5] * X * Z * Z +
                           a3[6] * Y * Y * Y + (Real)3 * a3[7] * Y * Y * Z +
                           (Real)3 * a3[8] * Y * Z * Z + a3[9] * Z * Z * Z;
        const Real tx = a3[0] + a3[3] + a3[5];
        const Real ty = a3[1] + a3[6] + a3[8];
        const Real tz = a3[2] + a3[7] + a3[9];
        const Real h3 = cubic - (Real)3 * (tx * X + ty * Y + tz * Z);
        G = G + h3 * (Real)(1.0 / 6.0);
    }
    return G;
}

constexpr int kL2DWarps = 8;

// Position of the k-th set bit (k >= 1) of m, which has at least k set bits.
__device__ __forceinline__ int nth_set_bit(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (c < k) {
            k -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Adjoint of DSMC2LB (the raw-coefficient mapping) at the listed nodes, one warp per node.
// With S and ppc fixed, every coefficient of the forward mapping is linear in the cell's
// cumulative sums M: c_0 = M_0 / (S ppc), and c_k = (M_k - s_k M_j) / (S ppc) where the
// forward subtracts s_k times the mean of component j (s_k M_0 for the diagonal second
// moments). The populations are f_q = w_q sum_k c_k B_k(xi_q) with the Hermite basis B of
// the forward series, so dL/dM = T^T (sum_q lam_q w_q B(xi_q)) / (S ppc). Lane l projects
// populations l and l + 32; the 20 projections are summed over the lanes by halving_sum.
// The forward overwrote the node's populations, so lam there is set to zero.
template <typename Real, class LAT>
__device__ __forceinline__ void d2l_adjoint_entries(const MapArgs<Real>& a, Real* lam,
                                                    double* grad_acc, int first, int stride) {
    const LatXi<LAT, Real>& lt = lat_xi<LAT, Real>();
    const unsigned lane = lane_id();
    const uint32_t S = a.ctrl[CTRL_NSAMPLES];
    for (int t = first; t < a.n; t += stride) {
        const int32_t node = a.list[t];
        if (node < 0 || (int64_t)node >= a.nnodes || S == 0) {
            if (lane == 0) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            continue;
        }
        const int x = node % a.nx, y = (node / a.nx) % a.ny - a.yh, z = node / (a.nx * a.ny);
        if (y < 0 || y >= a.ncy * a.lb_ratio) {
            if (lane == 0) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            continue;
        }
        const int64_t cell =
            ((int64_t)(z / a.lb_ratio) * a.ncy + y / a.lb_ratio) * a.ncx + (x / a.lb_ratio);
        Real v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = (Real)0;
#pragma unroll
        for (int h = 0; h < (LAT::Q + 31) / 32; ++h) {
            const int q = (int)lane + 32 * h;
            if (q < LAT::Q) {
                const int64_t at = (int64_t)q * a.nnodes + node;
                const Real lw = lam[at] * lt.w[q];
                lam[at] = (Real)0;
                const Real X = lt.x[3 * q], Y = lt.x[3 * q + 1], Z = lt.x[3 * q + 2];
                const Real hf = (Real)0.5;
                v[0] += lw;
                v[1] += lw * X;
                v[2] += lw * Y;
                v[3] += lw * Z;
                v[4] += lw * hf * (X * X - (Real)1);
                v[5] += lw * X * Y;
                v[6] += lw * X * Z;
                v[7] += lw * hf * (Y * Y - (Real)1);
                v[8] += lw * Y * Z;
                v[9] += lw * hf * (Z * Z - (Real)1);
                if (LAT::ORDER >= 3) {
                    const Real s6 = (Real)(1.0 / 6.0);
                    v[10] += lw * s6 * (X * X * X - (Real)3 * X);
                    v[11] += lw * hf * (X * X * Y - Y);
                    v[12] += lw * hf * (X * X * Z - Z);
                    v[13] += lw * hf * (X * Y * Y - X);
                    v[14] += lw * X * Y * Z;
                    v[15] += lw * hf * (X * Z * Z - X);
                    v[16] += lw * s6 * (Y * Y * Y - (Real)3 * Y);
                    v[17] += lw * hf * (Y * Y * Z - Z);
                    v[18] += lw * hf * (Y * Z * Z - Y);
                    v[19] += lw * s6 * (Z * Z * Z - (Real)3 * Z);
                }
            }
        }
        halving_sum<Real, 32>(v, lane);  // lane k holds projection k
        const double gk = (double)v[0];
        auto g = [&](int k) { return __shfl_sync(kFull, gk, k); };
        double d = gk;
        const double c0 = g(4) + g(7) + g(9);
        const double c1 = 3.0 * g(10) + g(13) + g(15);
        const double c2 = g(11) + 3.0 * g(16) + g(18);
        const double c3 = g(12) + g(17) + 3.0 * g(19);
        if (lane == 0) d -= c0;
        if (lane == 1) d -= c1;
        if (lane == 2) d -= c2;
        if (lane == 3) d -= c3;
        if (lane < (unsigned)kMoments) {
            double inv = 1.0 / ((double)S * (double)a.ppc);
            atomicAdd(&grad_acc[cell * kMoments + lane], d * inv);
        }
    }
}

template <typename Real, class LAT>
__global__ void __launch_bounds__(128) k_d2l_adj(MapArgs<Real> a, Real* lam, double* grad_acc) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    d2l_adjoint_entries<Real, LAT>(a, lam, grad_acc, (int)gw,
                                   (int)(((int64_t)gridDim.x * blockDim.x) >> 5));
}

// Raw Hermite basis of each lattice speed in FP64, for the LB2DSMC coefficient solve:
// B[q] = (1, xi_x, xi_y, xi_z, xi_i xi_j (xx xy xz yy yz zz), xi_i xi_j xi_k (xxx xxy xxz xyy
// xyz xzz yyy yyz yzz zzz)), xi = r e formed in double, built at compile time.
template <class LAT>
struct LatBasis {
    double b[LAT::Q][kMoments];
};
template <class LAT>
constexpr LatBasis<LAT> make_basis() {
    LatBasis<LAT> t{};
    for (int a = 0; a < LAT::Q; ++a) {
        double x[3] = {};
        for (int i = 0; i < 3; ++i) x[i] = lat_r<LAT>() * (double)LatTab<LAT>::e(a, i);
        int o = 0;
        t.b[a][o++] = 1.0;
        for (int i = 0; i < 3; ++i) t.b[a][o++] = x[i];
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j) t.b[a][o++] = x[i] * x[j];
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j)
                for (int k = j; k < 3; ++k) t.b[a][o++] = x[i] * x[j] * x[k];
    }
    return t;
}
__device__ const LatBasis<D3Q39> g_basis39 = make_basis<D3Q39>();
__device__ const LatBasis<D3Q19> g_basis19 = make_basis<D3Q19>();

template <class LAT>
__device__ __forceinline__ const LatBasis<LAT>& lat_basis() {
    if constexpr (LAT::Q == 39)
        return g_basis39;
    else
        return g_basis19;
}

// Index pairs and triples of the packed second and third moments.
__device__ __forceinline__ void packed_pair(int k, int& i, int& j) {
    constexpr int P[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    i = P[k][0];
    j = P[k][1];
}
__device__ __forceinline__ int packed_pair_index(int i, int j) {
    if (i > j) {
        const int t = i;
        i = j;
        j = t;
    }
    return i == 0 ? j : (i == 1 ? 2 + j : 5);
}

// Table 1 step 1 for the cell `cell`, in FP64 (the Grad-coefficient solve), by the whole
// block of kL2DWarps warps: FP64 runs at a small fraction of the FP32 rate, so its work is
// spread over the SM's four schedulers.
//   1. thread q < Q: the cell-mean population f_q, the mean of the cell's lb_ratio^2 (3D: ^3)
//      nodes summed in FP64;
//   2. warp w, lane k < 20: the partial raw moment sum_q f_q B_k(xi_q) over the populations
//      q in [w QW, (w + 1) QW) (fused multiply-adds, q ascending);
//   3. warp 0, lane k: R_k, the sum of the warps' partials (w ascending), then one comoving
//      coefficient from the raw moments:
//        u_i = R_i / rho,
//        a2_ij = R_ij / rho - u_i u_j - d_ij                                 (= sum f c c / rho - d),
//        a3_ijk = (R_ijk - u_i R_jk - u_j R_ik - u_k R_ij) / rho + 2 u_i u_j u_k (= sum f c c c / rho),
//      c = xi - u, exact identities of the centred sums.
// Every thread of the block calls it. Returns, in the lanes of warp 0, the packed FP64 value
// (lane k < 20 holds value k: a2[6], a3[10], u[3], C = 1 + 30 M) and rho.
template <typename Real, class LAT, bool Z3>
__device__ __forceinline__ void grad_coefficients(const MapArgs<Real>& a, int cell, double& mine,
                                                  double& rho_out) {
    constexpr int Q = LAT::Q;
    constexpr int NM = LAT::ORDER >= 3 ? kMoments : 10;  // raw moments of the order
    constexpr int W = kL2DWarps;
    constexpr int QW = (Q + W - 1) / W;
    __shared__ double s_f[Q];
    __shared__ double s_part[W][kMoments];
    const int t = (int)threadIdx.x, w = t >> 5;
    const unsigned lane = lane_id();
    const int r = a.lb_ratio;
    const int ix = cell % a.ncx, iy = (cell / a.ncx) % a.ncy, iz = cell / (a.ncx * a.ncy);
    constexpr int KN = Z3 ? 8 : 4;  // lb_ratio <= 2
    const int nk = Z3 ? r * r * r : r * r;
    if (t < Q) {
        Real p[KN];
#pragma unroll
        for (int k = 0; k < KN; ++k) {
            p[k] = 0;
            if (k < nk) {
                const int dz = Z3 ? k / (r * r) : 0, dy = (k / r) % r, dx = k % r;
                const int64_t node =
                    ((int64_t)(iz * r + dz) * a.ny + (iy * r + dy + a.yh)) * a.nx + (ix * r + dx);
                p[k] = a.f[(int64_t)t * a.nnodes + node];
            }
        }
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < KN; ++k)
            if (k < nk) sum += (double)p[k];
        // nk is 1, 4 or 8: the product by its reciprocal is the exact quotient
        s_f[t] = sum * (nk == 1 ? 1.0 : (nk == 4 ? 0.25 : 0.125));
    }
    __syncthreads();
    if (lane < (unsigned)NM) {
        const LatBasis<LAT>& B = lat_basis<LAT>();
        const int qa = w * QW, qb = qa + QW < Q ? qa + QW : Q;
        double part = 0.0;
        for (int q = qa; q < qb; ++q) part = fma(s_f[q], B.b[q][lane], part);
        s_part[w][lane] = part;
    }
    __syncthreads();
    if (w != 0) return;
    double R = 0.0;
    if (lane < (unsigned)NM)
#pragma unroll
        for (int v = 0; v < W; ++v) R += s_part[v][lane];
    auto at = [&](int k) { return __shfl_sync(kFull, R, k); };
    const double rho = at(0);
    double inv = 0.0;
    if (lane == 0) inv = 1.0 / rho;  // one FP64 reciprocal, broadcast
    inv = __shfl_sync(kFull, inv, 0);
    const double u[3] = {at(1) * inv, at(2) * inv, at(3) * inv};
    double R2[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) R2[k] = at(4 + k);
    double val = 0.0;
    if (lane >= 4u && lane < 10u) {
        int i, j;
        packed_pair((int)lane - 4, i, j);
        val = R * inv - u[i] * u[j] - (i == j ? 1.0 : 0.0);
    } else if (lane >= 10u && lane < (unsigned)NM) {
        constexpr int T[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                  {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
        const int i = T[lane - 10u][0], j = T[lane - 10u][1], k = T[lane - 10u][2];
        const double cross = u[i] * R2[packed_pair_index(j, k)] + u[j] * R2[packed_pair_index(i, k)] +
                             u[k] * R2[packed_pair_index(i, j)];
        val = (R - cross) * inv + 2.0 * u[i] * u[j] * u[k];
    }
    // M = max |val| over the lanes: the bits of non-negative doubles order as unsigned integers
    // (a NaN coefficient is left out, as fmax does)
    unsigned long long mb = val == val ? (unsigned long long)__double_as_longlong(fabs(val)) : 0ull;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long ob = (unsigned long long)__shfl_xor_sync(kFull, (long long)mb, o);
        mb = ob > mb ? ob : mb;
    }
    const double M = __longlong_as_double((long long)mb);
    // packed values: lane k < 16 takes coefficient k (a2 at lanes 4-9, a3 at 10-19), lanes
    // 16-18 u, lane 19 C
    const double mv = __shfl_sync(kFull, val, (int)(lane + 4u) & 31);
    mine = lane < (unsigned)(NM - 4) ? mv : 0.0;
    if (lane == GR_U) mine = u[0];
    if (lane == GR_U + 1) mine = u[1];
    if (lane == GR_U + 2) mine = u[2];
    if (lane == GR_C) mine = 1.0 + 30.0 * M;
    rho_out = rho;
}

// LB2DSMC for the listed cells: one block per cell (see the top of this file). An invalid
// cell index is skipped and flagged; a cell whose new count exceeds its bin keeps its
// particles and raises the capacity status. The Grad record of each listed cell is written
// to a.grad.
// MOVE (the fused multi-step pass): the listed cells' particles were left in the half of
// x.. (counts `count`) by the fused pass, the new particles are moved on at once (the move of
// the next step, keyed like the particle's slot) into the bins of the half of ax.. with their
// order keys, and a kept cell's particles are moved on likewise.
template <typename Real, bool Z3>
__device__ __forceinline__ MoveCtx<Real> l2d_move_ctx(const MapArgs<Real>& a) {
    MoveCtx<Real> m;
    m.H = (Real)a.ncx;
    // the fused pass (and so this move) runs on contexts that hold the whole channel
    m.L = (Real)a.ncy;
    m.Lz = (Real)(a.ncz ? a.ncz : 1);
    m.dt = a.dt_r;
    m.g = a.g_r;
    m.ncx = a.ncx;
    m.ncy = a.ncy;
    m.y0 = 0;
    m.nly = a.ncy;
    m.ncz = a.ncz;
    m.bin = (uint32_t)a.bin;
    m.seed = a.seed;
    return m;
}

template <typename Real, class LAT, bool Z3, bool MOVE = false>
__device__ __forceinline__ void l2d_cells(const MapArgs<Real>& a, int first, int stride) {
    __shared__ unsigned s_am[kL2DWarps], s_em[kL2DWarps], s_vm[kL2DWarps];
    __shared__ Real s_c[20];
    __shared__ uint32_t s_nnew;
    const uint32_t t_step = a.ctrl[CTRL_STEP];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int w = threadIdx.x >> 5;
    const uint32_t bin = (uint32_t)a.bin;
    unsigned long long deleted = 0, created = 0, attempts = 0, envelope = 0;
    uint32_t flags = 0;
    int32_t dlive = 0;
    uint32_t hits = 0, caps = 0, lost = 0;  // moves of the fused pass
    const Half<Real> dst{a.arec, a.acount};
    for (int ci = first; ci < a.n; ci += stride) {
        const int32_t icell = a.list[ci];
        if (icell < 0 || icell >= a.ncx * a.ncy * (Z3 ? a.ncz : 1)) {
            flags |= HYB_ST_BAD_INPUT;
            continue;
        }
        const uint32_t cell = (uint32_t)icell;
        // the channel's cell: the key of the cell's random streams and of the stable order
        const uint32_t gcell = global_cell(cell, a.ncx, a.ncy, a.y0, a.ncy_g);
        const uint32_t old = threadIdx.x == 0 ? a.count[cell] : 0u;
        double mine = 0.0, rho = 0.0;
        grad_coefficients<Real, LAT, Z3>(a, icell, mine, rho);  // the block; results in warp 0
        if (w == 0) {
            GradRec& g = a.grad[ci];
            if (lane < 20u) {
                s_c[lane] = (Real)mine;  // the sampler takes its decisions in the state precision
                g.v[lane] = mine;
            }
            if (lane == 0) {
                const double ur = u01d(draw(a.seed, gcell, t_step, TAG_L2D_ROUND, 0, 0).x);
                const double ne = floor(rho * (double)a.ppc + ur);
                const uint32_t nnew = ne > 0.0 ? (uint32_t)ne : 0u;
                s_nnew = nnew;
                g.rho = rho;
                g.nnew = nnew;
                g.pad = 0;
            }
        }
        __syncthreads();
        const uint32_t nnew = s_nnew;
        Real a2[6], a3[10];
#pragma unroll
        for (int k = 0; k < 6; ++k) a2[k] = s_c[GR_A2 + k];
#pragma unroll
        for (int k = 0; k < 10; ++k) a3[k] = s_c[GR_A3 + k];
        const Real C = s_c[GR_C];
        const Real ux = s_c[GR_U], uy = s_c[GR_U + 1], uz = s_c[GR_U + 2];
        __syncthreads();  // s_c and s_nnew are rewritten for the next cell
        const int64_t out0 = (int64_t)cell * bin;
        if (nnew > bin) {  // the cell keeps its particles
            flags |= HYB_ST_CAPACITY;
            if constexpr (MOVE) {
                // ... and moves them on; the cell's count is read by every thread
                uint32_t nold = a.count[cell];
                if (nold > bin) nold = bin;
                const MoveCtx<Real> m = l2d_move_ctx<Real, Z3>(a);
                for (uint32_t k0 = 0; k0 < nold; k0 += kL2DWarps * 32) {
                    const uint32_t k = k0 + threadIdx.x;
                    const bool act = k < nold;
                    Real px = 0, py = 0, pz = 0, ux = 0, uy = 0, uz = 0;
                    uint32_t key = 0, tg, ok = 0;
                    if (act) {
                        rec_get(a.rec, out0 + k, px, py, pz, ux, uy, uz, tg);
                        int dir;
                        key = move_particle<Real, Z3>(m, origin_of(m, gcell), k, t_step, px, py, pz, ux, uy,
                                                      uz, hits, caps, dir, ok);
                    }
                    const uint32_t arr = bin_arrival1(dst.count, key, act, lane);
                    if (act) {
                        if (arr < bin)
                            put_particle<Real, Z3>(dst, (int64_t)key * bin + arr, ok, px, py, pz, ux, uy, uz);
                        else
                            lost += 1;
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) a.count[cell] = 0;
            }
            continue;
        }
        const Real fx = (Real)(cell % (uint32_t)a.ncx);
        const Real fy = (Real)(a.y0 + (int)((cell / (uint32_t)a.ncx) % (uint32_t)a.ncy));
        const Real fz = Z3 ? (Real)(cell / ((uint32_t)a.ncx * (uint32_t)a.ncy)) : (Real)0;
        const uint64_t cap64 = 1000ull * nnew;
        const uint32_t cap = cap64 < 0xFFFFFFull ? (uint32_t)cap64 : 0xFFFFFFu;
        uint32_t produced = 0, j0 = 0;
        while (produced < nnew && j0 < cap) {
            const uint32_t j = j0 + threadIdx.x;
            const bool valid = j < cap;
            bool acc = false, env = false;
            Real X = 0, Y = 0, Z = 0;
            uint4 r2 = make_uint4(0u, 0u, 0u, 0u);
            if (valid) {
                const uint4 r1 = draw(a.seed, gcell, t_step, TAG_L2D_VEL, j, 0);
                r2 = draw(a.seed, gcell, t_step, TAG_L2D_VEL, j, 1);
                Real spare;
                gauss_pair<Real>(r1.x, r1.y, X, Y);
                gauss_pair<Real>(r1.z, r1.w, Z, spare);
                const Real G = grad_G<Real, LAT::ORDER>(a2, a3, X, Y, Z);
                const Real R = (Real)u01f(r2.x);
                env = G > C;
                acc = C * R <= G;
            }
            const unsigned am = __ballot_sync(kFull, acc);
            const unsigned em = __ballot_sync(kFull, env);
            const unsigned vm = __ballot_sync(kFull, valid);
            if (lane == 0) {
                s_am[w] = am;
                s_em[w] = em;
                s_vm[w] = vm;
            }
            __syncthreads();
            uint32_t before = 0, total = 0;
#pragma unroll
            for (int v = 0; v < kL2DWarps; ++v) {
                const uint32_t cv = (uint32_t)__popc(s_am[v]);
                if (v < w) before += cv;
                total += cv;
            }
            const uint32_t need = nnew - produced;
            const uint32_t rank = before + (uint32_t)__popc(am & lt);
            if constexpr (MOVE) {
                // the new particle of slot produced + rank, moved on at once
                const bool mk = acc && rank < need;
                const uint32_t k = produced + rank;
                Real px = 0, py = 0, pz = 0, vx = 0, vy = 0, vz = 0;
                uint32_t key = 0, ok = 0;
                if (mk) {
                    px = fx + (Real)u01f(r2.y);
                    py = fy + (Real)u01f(r2.z);
                    if constexpr (Z3) pz = fz + (Real)u01f(r2.w);
                    vx = X + ux;
                    vy = Y + uy;
                    vz = Z + uz;
                    int dir;
                    const MoveCtx<Real> m = l2d_move_ctx<Real, Z3>(a);
                    key = move_particle<Real, Z3>(m, origin_of(m, gcell), k, t_step, px, py, pz, vx, vy, vz,
                                                  hits, caps, dir, ok);
                }
                const uint32_t arr = bin_arrival1(dst.count, key, mk, lane);
                if (mk) {
                    if (arr < bin)
                        put_particle<Real, Z3>(dst, (int64_t)key * bin + arr, ok, px, py, pz, vx, vy, vz);
                    else
                        lost += 1;
                }
            } else if (acc && rank < need) {
                const int64_t slot = out0 + produced + rank;
                rec_put(a.rec, slot, fx + (Real)u01f(r2.y), fy + (Real)u01f(r2.z),
                        Z3 ? fz + (Real)u01f(r2.w) : (Real)0, X + ux, Y + uy, Z + uz, 0u);
            }
            if (w == 0) {
                // trials consumed this round (up to the need-th accepted one, or all valid
                // ones) and envelope violations among them; lane v looks at warp v's trials
                const unsigned amv = lane < (unsigned)kL2DWarps ? s_am[lane] : 0u;
                const unsigned emv = lane < (unsigned)kL2DWarps ? s_em[lane] : 0u;
                const unsigned vmv = lane < (unsigned)kL2DWarps ? s_vm[lane] : 0u;
                const uint32_t cv = (uint32_t)__popc(amv);
                uint32_t inc = cv;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, inc, o);
                    if (lane >= (unsigned)o) inc += t;
                }
                const uint32_t exc = inc - cv;
                uint32_t mu = (uint32_t)__popc(vmv), me = (uint32_t)__popc(emv & vmv);
                if (total >= need) {
                    const unsigned last = __ballot_sync(kFull, exc < need && need <= inc);
                    const unsigned vl = (unsigned)(__ffs(last) - 1);
                    if (lane == vl) {
                        const int bit = nth_set_bit(amv, (int)(need - exc));
                        const unsigned upto = bit == 31 ? 0xFFFFFFFFu : ((2u << bit) - 1u);
                        mu = (uint32_t)bit + 1u;
                        me = (uint32_t)__popc(emv & upto);
                    } else if (lane > vl) {
                        mu = 0;
                        me = 0;
                    }
                }
                const uint32_t used = __reduce_add_sync(kFull, mu);
                const uint32_t envc = __reduce_add_sync(kFull, me);
                if (lane == 0) {
                    attempts += used;
                    envelope += envc;
                }
            }
            produced += min(total, need);
            j0 += kL2DWarps * 32;
            __syncthreads();
        }
        if (produced < nnew) flags |= HYB_ST_SAMPLING_CAP;
        if (threadIdx.x == 0) {
            deleted += old;
            created += produced;
            dlive += (int32_t)produced - (int32_t)old;
            // the fused pass's cell is consumed: its half's count starts the next arrivals
            a.count[cell] = MOVE ? 0u : produced;
        }
    }
    if constexpr (MOVE) move_events(a.counters, a.ctrl, hits, caps, lost, lane);
    flags = __reduce_or_sync(kFull, flags);
    if (threadIdx.x == 0) {
        if (deleted) atomicAdd(&a.counters[HYB_C_DELETED], deleted);
        if (created) atomicAdd(&a.counters[HYB_C_CREATED], created);
        if (attempts) atomicAdd(&a.counters[HYB_C_L2D_ATTEMPTS], attempts);
        if (envelope) atomicAdd(&a.counters[HYB_C_ENVELOPE], envelope);
        if (dlive) atomicAdd(&a.ctrl[CTRL_NTOT], (uint32_t)dlive);
    }
    if (lane == 0 && flags) atomicOr(&a.ctrl[CTRL_STATUS], flags);
}

// LB2DSMC: one block per listed cell (the listed cells of all replicas in the batch form).
template <typename Real, class LAT, bool BATCH, bool Z3 = false, bool MOVE = false>
__global__ void __launch_bounds__(kL2DWarps * 32) k_l2d(Launch<MapArgs<Real>> L) {
    pdl_begin();
    if constexpr (BATCH) {
        const int r = replica_of(L.pre, L.nrep, (int64_t)blockIdx.x);
        const MapArgs<Real>& a = L.tab[r];
        l2d_cells<Real, LAT, Z3, MOVE>(a, (int)(blockIdx.x - L.pre[r]), a.n);
    } else {
        l2d_cells<Real, LAT, Z3, MOVE>(L.one, (int)blockIdx.x, (int)gridDim.x);
    }
}

template <typename Real>
MapArgs<Real> map_args(Ctx& c, const int32_t* list, int32_t n) {
    MapArgs<Real> a{};
    a.f = (Real*)c.st.f[c.cur_f];
    a.nx = (int32_t)c.d.nx;
    a.ny = (int32_t)c.d.ny;
    a.ncx = c.p.ncx;
    a.ncy = c.p.ncy;
    a.lb_ratio = c.p.lb_ratio;
    a.ppc = c.p.ppc;
    a.n = n;
    a.bin = c.d.bin;
    a.nnodes = c.d.nnodes;
    a.list = list;
    a.eq_mode = c.p.d2l_mode;
    a.r_lat = c.d.r_lat;
    a.seed = c.p.seed;
    a.acc = c.st.acc;
    a.ctrl = c.st.ctrl;
    a.counters = c.st.counters;
    a.grad = c.st.grad;
    a.count = c.st.count[c.cur_p];
    a.rec = (Real*)c.st.part[c.cur_p];
    a.ncz = c.p.ncz >= 2 ? c.p.ncz : 0;
    a.y0 = c.p.ncy_global > 0 ? c.p.y0 : 0;
    a.ncy_g = c.p.ncy_global > 0 ? c.p.ncy_global : c.p.ncy;
    a.yh = (int32_t)c.d.yh;
    return a;
}

int blocks_for(const Ctx& c, int64_t threads_needed, int block, int per_sm) {
    int64_t b = (threads_needed + block - 1) / block;
    if (b > (int64_t)c.num_sms * per_sm) b = (int64_t)c.num_sms * per_sm;
    return (int)(b < 1 ? 1 : b);
}

template <typename Real, class LAT>
cudaError_t d2l_impl(Ctx& c, const int32_t* nodes, int32_t n) {
    MapArgs<Real> a = map_args<Real>(c, nodes, n);
    prof_begin(c, K_D2L);
    Launch<MapArgs<Real>> L{};
    L.one = a;
    L.total = n;
    const cudaError_t e = launch_pdl(k_d2l<Real, LAT, false>, dim3(blocks_for(c, (int64_t)n * 32, 128, 16)),
                                     dim3(128), 0, c.stream, L);
    prof_end(c, K_D2L);
    return e;
}

template <typename Real, class LAT>
cudaError_t l2d_launch(Ctx& c, const MapArgs<Real>& a, int32_t n) {
    prof_begin(c, K_L2D);
    Launch<MapArgs<Real>> L{};
    L.one = a;
    L.total = n;
    const dim3 grid(blocks_for(c, (int64_t)n * 32 * kL2DWarps, 32 * kL2DWarps, 8));
    const cudaError_t e =
        a.ncz ? launch_pdl(k_l2d<Real, LAT, false, true>, grid, dim3(32 * kL2DWarps), 0, c.stream, L)
              : launch_pdl(k_l2d<Real, LAT, false, false>, grid, dim3(32 * kL2DWarps), 0, c.stream, L);
    prof_end(c, K_L2D);
    return e;
}

template <typename Real, class LAT>
cudaError_t l2d_impl(Ctx& c, const int32_t* cells, int32_t n) {
    return l2d_launch<Real, LAT>(c, map_args<Real>(c, cells, n), n);
}

// LB2DSMC of the fused pass of parity p: the listed cells' particles are in half p^1, the
// moved particles go to half p.
template <typename Real, class LAT>
cudaError_t l2d_move_impl(Ctx& c, const int32_t* cells, int32_t n, int p) {
    const int save = c.cur_p;
    c.cur_p = p ^ 1;
    MapArgs<Real> a = map_args<Real>(c, cells, n);
    c.cur_p = save;
    a.arec = (Real*)c.st.part[p];
    a.acount = c.st.count[p];
    a.dt_r = (Real)c.d.dt;
    a.g_r = (Real)c.d.g_step;
    prof_begin(c, K_L2D);
    Launch<MapArgs<Real>> L{};
    L.one = a;
    L.total = n;
    const dim3 grid(blocks_for(c, (int64_t)n * 32 * kL2DWarps, 32 * kL2DWarps, 8));
    const cudaError_t e =
        a.ncz ? launch_pdl(k_l2d<Real, LAT, false, true, true>, grid, dim3(32 * kL2DWarps), 0, c.stream, L)
              : launch_pdl(k_l2d<Real, LAT, false, false, true>, grid, dim3(32 * kL2DWarps), 0, c.stream, L);
    prof_end(c, K_L2D);
    return e;
}

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
GradRec* g_scratch_addr[kMaxDevices] = {};

// Device address of the fixed scratch on `device`, which must be the current device. A
// __device__ array's address belongs to the CUDA context that loaded the module, so it is
// looked up again on every call whose stream is not being captured (a call after
// cudaDeviceReset, or from another context on the same device, gets its own context's
// address); during a capture the address of the last lookup on that device is used, which is
// why the first call on a device must come before any capture. The lock serialises
// concurrent first calls from several host threads.
cudaError_t noalloc_scratch(int device, cudaStream_t stream, GradRec** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_l2d_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = (GradRec*)p;
    }
    if (!g_scratch_addr[device]) return cudaErrorStreamCaptureUnsupported;
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

template <typename Real, class LAT>
cudaError_t l2d_noalloc_impl(Ctx& c, const int32_t* cells, int32_t n, GradRec* rec) {
    MapArgs<Real> a = map_args<Real>(c, cells, n);
    a.grad = rec;  // the fixed array instead of the arena's records
    return l2d_launch<Real, LAT>(c, a, n);
}

}  // namespace

namespace {
// The cumulative moment sums of the listed cells, in list order (zeros for an index out of
// range): one thread per value.
__global__ void k_gather_acc(const double* __restrict__ acc, const int32_t* __restrict__ cells,
                             int32_t n, int64_t ncells, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * kMoments) return;
    const int32_t c = cells[i / kMoments];
    out[i] = (c >= 0 && (int64_t)c < ncells) ? acc[(int64_t)c * kMoments + i % kMoments] : 0.0;
}
}  // namespace

cudaError_t launch_gather_acc(Ctx& c, const int32_t* cells, int32_t n, double* out) {
    const int64_t total = (int64_t)n * kMoments;
    k_gather_acc<<<(unsigned)((total + 255) / 256), 256, 0, c.stream>>>(c.st.acc, cells, n,
                                                                        c.d.ncells, out);
    return cudaGetLastError();
}

namespace {
// The coupling lists read from page-locked host memory (device-addressable) into the
// device staging: one thread per entry.
__global__ void k_lists_in(const int32_t* __restrict__ hn, int32_t nn, const int32_t* __restrict__ hc,
                           int32_t nc, int32_t* __restrict__ dn, int32_t* __restrict__ dc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nn)
        dn[i] = hn[i];
    else if (i < (int64_t)nn + nc)
        dc[i - nn] = hc[i - nn];
}

// The listed cells' moment sums (as k_gather_acc) and the status word, written straight to
// page-locked host memory.
__global__ void k_results_out(const double* __restrict__ acc, const int32_t* __restrict__ cells,
                              int32_t n, int64_t ncells, const uint32_t* __restrict__ status,
                              double* __restrict__ out, uint32_t* __restrict__ status_out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *status_out = *status;
    if (i >= (int64_t)n * kMoments) return;
    const int32_t c = cells[i / kMoments];
    out[i] = (c >= 0 && (int64_t)c < ncells) ? acc[(int64_t)c * kMoments + i % kMoments] : 0.0;
}
}  // namespace

cudaError_t launch_lists_in(Ctx& c, const int32_t* hn, int32_t nn, const int32_t* hc, int32_t nc,
                            int32_t* dn, int32_t* dc) {
    const int64_t total = (int64_t)nn + nc;
    if (total == 0) return cudaSuccess;
    k_lists_in<<<(unsigned)((total + 255) / 256), 256, 0, c.stream>>>(hn, nn, hc, nc, dn, dc);
    return cudaGetLastError();
}

cudaError_t launch_results_out(Ctx& c, const int32_t* cells, int32_t n, double* out,
                               uint32_t* status_out) {
    const int64_t total = (int64_t)n * kMoments;
    const unsigned grid = total > 0 ? (unsigned)((total + 255) / 256) : 1u;
    k_results_out<<<grid, 256, 0, c.stream>>>(c.st.acc, cells, n, c.d.ncells, c.st.ctrl + CTRL_STATUS,
                                              out, status_out);
    return cudaGetLastError();
}

cudaError_t launch_map_l2d_move(Ctx& c, const int32_t* cells, int32_t n, int p) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? l2d_move_impl<float, D3Q39>(c, cells, n, p)
                                   : l2d_move_impl<double, D3Q39>(c, cells, n, p);
    return c.p.real_bytes == 4 ? l2d_move_impl<float, D3Q19>(c, cells, n, p)
                               : l2d_move_impl<double, D3Q19>(c, cells, n, p);
}

cudaError_t launch_map_l2d_noalloc(Ctx& c, const int32_t* cells, int32_t n) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != c.device) return cudaErrorInvalidDevice;
    GradRec* rec = nullptr;
    e = noalloc_scratch(dev, c.stream, &rec);
    if (e != cudaSuccess) return e;
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? l2d_noalloc_impl<float, D3Q39>(c, cells, n, rec)
                                   : l2d_noalloc_impl<double, D3Q39>(c, cells, n, rec);
    return c.p.real_bytes == 4 ? l2d_noalloc_impl<float, D3Q19>(c, cells, n, rec)
                               : l2d_noalloc_impl<double, D3Q19>(c, cells, n, rec);
}

size_t map_args_bytes(int real_bytes) {
    return real_bytes == 4 ? sizeof(MapArgs<float>) : sizeof(MapArgs<double>);
}

void map_args_fill(Ctx& c, int cur_p, int cur_f, const int32_t* list, int32_t n, void* out) {
    const int sp = c.cur_p, sf = c.cur_f;
    c.cur_p = cur_p;
    c.cur_f = cur_f;
    if (c.p.real_bytes == 4) {
        const MapArgs<float> a = map_args<float>(c, list, n);
        std::memcpy(out, &a, sizeof(a));
    } else {
        const MapArgs<double> a = map_args<double>(c, list, n);
        std::memcpy(out, &a, sizeof(a));
    }
    c.cur_p = sp;
    c.cur_f = sf;
}

namespace {
template <typename Real, class LAT>
cudaError_t batch_d2l_impl(BatchDev& b, int cur_p, int cur_f) {
    Launch<MapArgs<Real>> L{};
    L.tab = (const MapArgs<Real>*)b.d2l[cur_p][cur_f];
    L.pre = b.pre_d2l;
    L.nrep = b.nrep;
    L.total = b.tot_d2l;
    const int64_t blocks = (b.tot_d2l * 32 + b.d2l_block - 1) / b.d2l_block;
    return launch_pdl(k_d2l<Real, LAT, true>, dim3((unsigned)blocks), dim3(b.d2l_block), 0, b.stream, L);
}

template <typename Real, class LAT>
cudaError_t batch_l2d_impl(BatchDev& b, int cur_p, int cur_f) {
    Launch<MapArgs<Real>> L{};
    L.tab = (const MapArgs<Real>*)b.l2d[cur_p][cur_f];
    L.pre = b.pre_l2d;
    L.nrep = b.nrep;
    L.total = b.tot_l2d;
    return launch_pdl(k_l2d<Real, LAT, true>, dim3((unsigned)b.tot_l2d), dim3(32 * kL2DWarps), 0, b.stream, L);
}
}  // namespace

cudaError_t launch_batch_d2l(BatchDev& b, int cur_p, int cur_f) {
    if (b.lattice == 39)
        return b.real_bytes == 4 ? batch_d2l_impl<float, D3Q39>(b, cur_p, cur_f)
                                 : batch_d2l_impl<double, D3Q39>(b, cur_p, cur_f);
    return b.real_bytes == 4 ? batch_d2l_impl<float, D3Q19>(b, cur_p, cur_f)
                             : batch_d2l_impl<double, D3Q19>(b, cur_p, cur_f);
}

cudaError_t launch_batch_l2d(BatchDev& b, int cur_p, int cur_f) {
    if (b.lattice == 39)
        return b.real_bytes == 4 ? batch_l2d_impl<float, D3Q39>(b, cur_p, cur_f)
                                 : batch_l2d_impl<double, D3Q39>(b, cur_p, cur_f);
    return b.real_bytes == 4 ? batch_l2d_impl<float, D3Q19>(b, cur_p, cur_f)
                             : batch_l2d_impl<double, D3Q19>(b, cur_p, cur_f);
}

namespace {
template <typename Real, class LAT>
cudaError_t d2l_adj_impl(Ctx& c, const int32_t* nodes, int32_t n, void* lam, double* grad_acc) {
    const MapArgs<Real> a = map_args<Real>(c, nodes, n);
    k_d2l_adj<Real, LAT><<<blocks_for(c, (int64_t)n * 32, 128, 16), 128, 0, c.stream>>>(
        a, (Real*)lam, grad_acc);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_map_d2l_adjoint(Ctx& c, const int32_t* nodes, int32_t n, void* lam,
                                   double* grad_acc) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? d2l_adj_impl<float, D3Q39>(c, nodes, n, lam, grad_acc)
                                   : d2l_adj_impl<double, D3Q39>(c, nodes, n, lam, grad_acc);
    return c.p.real_bytes == 4 ? d2l_adj_impl<float, D3Q19>(c, nodes, n, lam, grad_acc)
                               : d2l_adj_impl<double, D3Q19>(c, nodes, n, lam, grad_acc);
}

cudaError_t launch_map_d2l(Ctx& c, const int32_t* nodes, int32_t n) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? d2l_impl<float, D3Q39>(c, nodes, n) : d2l_impl<double, D3Q39>(c, nodes, n);
    return c.p.real_bytes == 4 ? d2l_impl<float, D3Q19>(c, nodes, n) : d2l_impl<double, D3Q19>(c, nodes, n);
}

cudaError_t launch_map_l2d(Ctx& c, const int32_t* cells, int32_t n) {
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? l2d_impl<float, D3Q39>(c, cells, n) : l2d_impl<double, D3Q39>(c, cells, n);
    return c.p.real_bytes == 4 ? l2d_impl<float, D3Q19>(c, cells, n) : l2d_impl<double, D3Q19>(c, cells, n);
}

}  // namespace hyb
