// Oracle: the two kinetic mappings of Sec. 2.
//
// TEST INFRASTRUCTURE ONLY (see ora_common.hpp).
//
// DSMC2LB (Sec. 2.1): the cumulative DSMC sums of a cell give rho, u and the raw second and
// third velocity moments; these give the Hermite coefficients a^(n) (Eq. nordercoefficients
// with f the particle distribution), and the populations at the coupling node are
// f_a = w_a sum_{n<=N} a^(n) : H^(n)(xi_a) / n!  (Eq. discretefunctions).
//
// LB2DSMC (Sec. 2.2, Table 1): from the populations, rho and u, then the Grad coefficients
// of the distribution in the frame moving with u, normalised by rho (so a^(0) = 1 and
// a^(1) = 0, and G of Eq. distr_outeq starts at n = 2): a2_ij = sum f c_i c_j / rho - d_ij,
// a3_ijk = sum f c_i c_j c_k / rho with c = xi_a - u, in FP64. M = largest |component|,
// C = 1 + 30 M (Eq. C). Trial velocities from the unit Maxwellian by Box-Muller, accepted
// when C R <= G(xi), taken in the state precision with the coefficients rounded to it; the
// particle velocity is sqrt(kT/m) xi + u, i.e.
// xi + u in c_th units (Eq. step6 read with the unit-variance weight of Eq. globalMax). The
// particle count conserves the mapped mass: E[N] = rho * ppc, rounded stochastically.
#pragma once
#include "ora_dsmc.hpp"
#include "ora_lbm.hpp"

namespace ora {

constexpr int kMaxL2DAttempts = 1000;

// Index of the packed symmetric moment for (i <= j) and (i <= j <= k), in the sampling order.
inline int packed2(int i, int j) {
    int o = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++o)
            if (a == i && b == j) return o;
    return -1;
}
inline int packed3(int i, int j, int k) {
    int o = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b)
            for (int e = b; e < 3; ++e, ++o)
                if (a == i && b == j && e == k) return o;
    return -1;
}
inline void sort3(int& a, int& b, int& c) {
    if (a > b) std::swap(a, b);
    if (b > c) std::swap(b, c);
    if (a > b) std::swap(a, b);
}

// Raw Hermite coefficients of a cell from its cumulative sums (S samples).
inline bool dsmc_coefficients(const double* m, uint64_t S, int ppc, Coeffs& a) {
    const double NS = m[0];
    if (S == 0 || !(NS > 0.0)) return false;
    const double rho = (NS / (double)S) / (double)ppc;
    double m1[3], m2[3][3], m3[3][3][3];
    for (int i = 0; i < 3; ++i) m1[i] = m[1 + i] / NS;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int a2 = std::min(i, j), b2 = std::max(i, j);
            m2[i][j] = m[4 + packed2(a2, b2)] / NS;
            for (int k = 0; k < 3; ++k) {
                int x = i, y = j, z = k;
                sort3(x, y, z);
                m3[i][j][k] = m[10 + packed3(x, y, z)] / NS;
            }
        }
    a = Coeffs{};
    a.a0 = rho;
    for (int i = 0; i < 3; ++i) {
        a.a1[i] = rho * m1[i];
        for (int j = 0; j < 3; ++j) {
            a.a2[i][j] = rho * (m2[i][j] - kd(i, j));
            for (int k = 0; k < 3; ++k)
                a.a3[i][j][k] = rho * (m3[i][j][k] - m1[i] * kd(j, k) - m1[j] * kd(i, k) -
                                       m1[k] * kd(i, j));
        }
    }
    return true;
}

// Grad coefficients of Table 1 step 1, written out from their definition in FP64 (the
// precision the Grad solve takes), in the frame moving with u and normalised by rho, from
// the populations f[q] (q < L.q):
//   rho = sum_a f_a,  u_i = (sum_a f_a xi_ai) / rho,  c_a = xi_a - u,
//   a2_ij = (sum_a f_a c_ai c_aj) / rho - d_ij,  a3_ijk = (sum_a f_a c_ai c_aj c_ak) / rho,
// every sum taken over a in population order. M = largest |component| of a2 and a3 and
// C = 1 + 30 M (Eq. C).
struct GradCell {
    double rho;
    double u[3];
    Coeffs ahat;  // ahat.a0 = 1, a1 = 0
    double M, C;
};

inline GradCell grad_from_populations(const Lattice& L, const double* f, int order) {
    const int Q = L.q;
    GradCell g{};
    g.rho = 0.0;
    for (int q = 0; q < Q; ++q) g.rho += f[q];
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int q = 0; q < Q; ++q) s += f[q] * L.xi[q][i];
        g.u[i] = s / g.rho;
    }
    std::vector<std::array<double, 3>> c((size_t)Q);
    for (int q = 0; q < Q; ++q)
        for (int i = 0; i < 3; ++i) c[q][i] = L.xi[q][i] - g.u[i];
    g.ahat = Coeffs{};
    g.ahat.a0 = 1.0;
    double M = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int q = 0; q < Q; ++q) s += f[q] * c[q][i] * c[q][j];
            g.ahat.a2[i][j] = s / g.rho - kd(i, j);
            M = std::max(M, std::fabs(g.ahat.a2[i][j]));
            if (order < 3) continue;
            for (int k = 0; k < 3; ++k) {
                double s3 = 0.0;
                for (int q = 0; q < Q; ++q) s3 += f[q] * c[q][i] * c[q][j] * c[q][k];
                g.ahat.a3[i][j][k] = s3 / g.rho;
                M = std::max(M, std::fabs(g.ahat.a3[i][j][k]));
            }
        }
    g.M = M;
    g.C = 1.0 + 30.0 * M;
    return g;
}

// G of Eq. distr_outeq in the state precision, from the comoving coefficients packed by
// symmetry (a2: xx xy xz yy yz zz; a3: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz), as the full
// sums over i, j (, k) of Table 1 grouped by distinct entries:
//   a2 : H2 = sum_i a2_ii (x_i^2 - 1) + 2 sum_{i<j} a2_ij x_i x_j,
//   a3 : H3 = sum over distinct (i<=j<=k) of (multiplicity) a3_ijk x_i x_j x_k - 3 x . t,
//   t_i = sum_j a3_ijj. The grouping is fixed so that the accept decision is reproducible.
template <class Real>
Real grad_G(const Real* a2, const Real* a3, const Real* xi, int order) {
    const Real X = xi[0], Y = xi[1], Z = xi[2];
    const Real h2 = a2[0] * (X * X - (Real)1) + a2[3] * (Y * Y - (Real)1) +
                    a2[5] * (Z * Z - (Real)1) +
                    (Real)2 * (a2[1] * X * Y + a2[2] * X * Z + a2[4] * Y * Z);
    Real G = (Real)1 + (Real)0.5 * h2;
    if (order >= 3) {
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

// Packed state-precision copies of a cell's Grad coefficients.
template <class Real>
struct GradPacked {
    Real a2[6], a3[10], u[3], C;
};

// The FP64 coefficients packed by symmetry and rounded to the state precision Real, in which
// the sampler takes its accept decisions (Table 1 steps 4-6).
template <class Real>
GradPacked<Real> pack(const GradCell& g) {
    GradPacked<Real> p;
    const int i2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    const int i3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                           {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
    for (int k = 0; k < 6; ++k) p.a2[k] = (Real)g.ahat.a2[i2[k][0]][i2[k][1]];
    for (int k = 0; k < 10; ++k) p.a3[k] = (Real)g.ahat.a3[i3[k][0]][i3[k][1]][i3[k][2]];
    for (int i = 0; i < 3; ++i) p.u[i] = (Real)g.u[i];
    p.C = (Real)g.C;
    return p;
}

// Table 1 steps 4-6 for one cell: trials j = 0, 1, 2, ... of the cell's stream (Philox
// blocks 0 and 1 of counter (cell, t, tag, j)); a trial draws xi from the unit Maxwellian
// by Box-Muller and R uniform, and is accepted when C R <= G(xi). The k-th accepted trial
// gives the k-th new particle: velocity xi + u, position from the trial's block-1 words.
// Trials are capped at min(1000 n, 2^24); particles left without a trial are appended as
// deleted (x = -1). Returns the number of trials used.
template <class Real>
uint64_t grad_sample_cell(const GradPacked<Real>& g, int order, uint64_t seed, uint32_t cell,
                          uint32_t t, uint32_t n, Real ix, Real iy, Real iz, bool three_d,
                          Real* out /* n x 6: x y z vx vy vz */, uint64_t* envelope,
                          bool* capped) {
    const uint64_t cap = std::min<uint64_t>(1000ull * n, 0xFFFFFFull);
    uint32_t produced = 0;
    uint64_t j = 0;
    for (; produced < n && j < cap; ++j) {
        U4 r = draw(seed, cell, t, TAG_L2D_VEL, (uint32_t)j, 0);
        U4 r2 = draw(seed, cell, t, TAG_L2D_VEL, (uint32_t)j, 1);
        Real xi[3], spare;
        gauss_pair<Real>(r[0], r[1], xi[0], xi[1]);
        gauss_pair<Real>(r[2], r[3], xi[2], spare);
        const Real G = grad_G<Real>(g.a2, g.a3, xi, order);
        const Real R = (Real)u01f(r2[0]);
        if (G > g.C) *envelope += 1;
        if (g.C * R <= G) {
            Real* o = out + 6 * (size_t)produced;
            o[0] = ix + (Real)u01f(r2[1]);
            o[1] = iy + (Real)u01f(r2[2]);
            o[2] = three_d ? iz + (Real)u01f(r2[3]) : (Real)0;
            for (int i = 0; i < 3; ++i) o[3 + i] = xi[i] + g.u[i];
            produced += 1;
        }
    }
    *capped = produced < n;
    for (; produced < n; ++produced) {
        Real* o = out + 6 * (size_t)produced;
        o[0] = (Real)-1;
        o[1] = iy;
        o[2] = iz;
        o[3] = o[4] = o[5] = (Real)0;
    }
    return j;
}

template <class Real>
void map_dsmc_to_lbm(Dsmc<Real>& D, Lbm<Real>& B, const int32_t* nodes, int n) {
    const Lattice& L = B.L;
    for (int t = 0; t < n; ++t) {
        const int64_t node = nodes[t];
        if (node < 0 || node >= B.d.nnodes) {
            D.status |= ST_BAD_INPUT;
            continue;
        }
        // a streamwise slab's yh ghost rows below and above its rows hold no cell of its own
        const int64_t x = node % B.d.nx, y = (node / B.d.nx) % B.d.ny - B.d.yh;
        const int64_t z = node / (B.d.nx * B.d.ny);
        if (y < 0 || y >= (int64_t)D.p.ncy * D.p.lb_ratio) {
            D.status |= ST_BAD_INPUT;
            continue;
        }
        const int64_t zc = D.three_d() ? z / D.p.lb_ratio : 0;
        const int64_t cell = (zc * D.p.ncy + y / D.p.lb_ratio) * D.p.ncx + (x / D.p.lb_ratio);
        Coeffs a;
        if (!dsmc_coefficients(&D.acc[(size_t)cell * kNumMoments], D.nsamples, D.p.ppc, a)) {
            D.status |= ST_BAD_INPUT;
            continue;
        }
        if (D.p.d2l_mode == 1) {  // the local equilibrium of rho and u (Sec. 4, Eq. feq_dsmc)
            double u[3];
            for (int i = 0; i < 3; ++i) u[i] = a.a1[i] / a.a0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    a.a2[i][j] = a.a0 * u[i] * u[j];
                    for (int k = 0; k < 3; ++k) a.a3[i][j][k] = a.a0 * u[i] * u[j] * u[k];
                }
        }
        for (int q = 0; q < L.q; ++q)
            B.f[(size_t)q * B.d.nnodes + node] =
                (Real)(L.w[q] * hermite_series(a, L.xi[q].data(), B.d.order));
    }
}

// LB2DSMC over a list of distinct cells: each listed cell's particles are replaced by the
// cell's regenerated ones (Sec. 2.2: their number carries the mapped mass of the coupling
// site), so the particle array stays ordered by cell. A cell whose new count exceeds the
// per-cell slot count `bin` keeps its particles and raises the capacity status; an invalid
// cell index is skipped and raises the bad-input status.
template <class Real>
void map_lbm_to_dsmc(Dsmc<Real>& D, const Lbm<Real>& B, const int32_t* cells, int n) {
    const Lattice& L = B.L;
    const int r = D.p.lb_ratio;
    const uint32_t t = (uint32_t)D.step;
    std::vector<int> slot_of(D.d.ncells, -1);
    std::vector<std::vector<Real>> fresh(n);
    for (int c = 0; c < n; ++c) {
        if (cells[c] < 0 || cells[c] >= D.d.ncells) {  // skipped and flagged
            D.status |= ST_BAD_INPUT;
            continue;
        }
        const int64_t cell = cells[c];
        const int64_t ix = cell % D.p.ncx, iy = (cell / D.p.ncx) % D.p.ncy;
        const int64_t iz = cell / ((int64_t)D.p.ncx * D.p.ncy);
        const uint32_t gc = channel_cell(D.p, cell);  // the key of the cell's random streams
        const int64_t yh = B.d.yh;                    // a slab's ghost rows below its LB rows
        const int rz = D.three_d() ? r : 1;  // LB layers of the cell along z
        // the mean populations of the cell's nodes and its Grad coefficients, in FP64
        std::vector<double> fbar(L.q, 0.0);
        for (int q = 0; q < L.q; ++q) {
            double s = 0.0;
            for (int dz = 0; dz < rz; ++dz)
                for (int dy = 0; dy < r; ++dy)
                    for (int dx = 0; dx < r; ++dx)
                        s += (double)B.fa(q, ix * r + dx, iy * r + dy + yh, iz * rz + dz);
            fbar[q] = s / (double)(r * r * rz);
        }
        const GradCell g = grad_from_populations(L, fbar.data(), B.d.order);
        const double u = u01d(draw(D.p.seed, gc, t, TAG_L2D_ROUND, 0, 0)[0]);
        const double ne = std::floor(g.rho * (double)D.p.ppc + u);
        const uint32_t nnew = ne > 0.0 ? (uint32_t)ne : 0u;
        if (nnew > (uint32_t)D.d.bin) {
            D.status |= ST_CAPACITY;
            continue;
        }
        fresh[c].resize(6 * (size_t)nnew);
        bool capped = false;
        const uint64_t trials = grad_sample_cell<Real>(pack<Real>(g), B.d.order, D.p.seed, gc, t,
                                                       nnew, (Real)ix, (Real)(D.y0() + iy),
                                                       (Real)iz, D.three_d(), fresh[c].data(),
                                                       &D.counters[C_ENVELOPE], &capped);
        if (capped) D.status |= ST_SAMPLING_CAP;
        D.counters[C_L2D_ATTEMPTS] += trials;
        D.counters[C_CREATED] += nnew;
        D.counters[C_DELETED] += D.cell_start[cell + 1] - D.cell_start[cell];
        slot_of[cell] = c;
    }
    const bool td = D.three_d();
    std::vector<Real> nx, ny, nz, nvx, nvy, nvz;
    std::vector<uint32_t> cs(D.d.ncells + 1, 0);
    for (int64_t cell = 0; cell < D.d.ncells; ++cell) {
        cs[cell] = (uint32_t)nx.size();
        if (slot_of[cell] >= 0) {
            const std::vector<Real>& o = fresh[slot_of[cell]];
            for (size_t k = 0; k < o.size() / 6; ++k) {
                nx.push_back(o[6 * k]);
                ny.push_back(o[6 * k + 1]);
                if (td) nz.push_back(o[6 * k + 2]);
                nvx.push_back(o[6 * k + 3]);
                nvy.push_back(o[6 * k + 4]);
                nvz.push_back(o[6 * k + 5]);
            }
        } else {
            for (uint32_t i = D.cell_start[cell]; i < D.cell_start[cell + 1]; ++i) {
                nx.push_back(D.x[i]);
                ny.push_back(D.y[i]);
                if (td) nz.push_back(D.z[i]);
                nvx.push_back(D.vx[i]);
                nvy.push_back(D.vy[i]);
                nvz.push_back(D.vz[i]);
            }
        }
    }
    cs[D.d.ncells] = (uint32_t)nx.size();
    D.x.swap(nx);
    D.y.swap(ny);
    D.z.swap(nz);
    D.vx.swap(nvx);
    D.vy.swap(nvy);
    D.vz.swap(nvz);
    D.cell_start.swap(cs);
}

}  // namespace ora
