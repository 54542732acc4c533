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
// a3_ijk = sum f c_i c_j c_k / rho with c = xi_a - u. M = largest |component|, C = 1 + 30 M
// (Eq. C). Trial velocities from the unit Maxwellian by Box-Muller, accepted when
// C R <= G(xi); the particle velocity is sqrt(kT/m) xi + u, i.e. xi + u in c_th units
// (Eq. step6 read with the unit-variance weight of Eq. globalMax). The particle count
// conserves the mapped mass: E[N] = rho * ppc, rounded stochastically.
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

// Grad coefficients in the comoving frame, normalised by rho (Table 1 step 1).
struct GradCell {
    double rho;
    double u[3];
    Coeffs ahat;  // ahat.a0 = 1, a1 = 0
    double M, C;
};

inline GradCell grad_from_populations(const Lattice& L, const double* f, int order) {
    GradCell g{};
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int a = 0; a < L.q; ++a) {
        rho += f[a];
        for (int i = 0; i < 3; ++i) j[i] += f[a] * L.xi[a][i];
    }
    g.rho = rho;
    for (int i = 0; i < 3; ++i) g.u[i] = j[i] / rho;
    Coeffs& h = g.ahat;
    h = Coeffs{};
    h.a0 = 1.0;
    for (int a = 0; a < L.q; ++a) {
        double c[3];
        for (int i = 0; i < 3; ++i) c[i] = L.xi[a][i] - g.u[i];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                h.a2[i][k] += f[a] * c[i] * c[k] / rho;
                if (order >= 3)
                    for (int l = 0; l < 3; ++l) h.a3[i][k][l] += f[a] * c[i] * c[k] * c[l] / rho;
            }
    }
    for (int i = 0; i < 3; ++i) h.a2[i][i] -= 1.0;
    double M = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            M = std::max(M, std::fabs(h.a2[i][k]));
            for (int l = 0; l < 3; ++l) M = std::max(M, std::fabs(h.a3[i][k][l]));
        }
    g.M = M;
    g.C = 1.0 + 30.0 * M;
    return g;
}

// One accepted velocity (Table 1 steps 4-6) for particle k of cell `cell` at step t.
// Returns the number of attempts (> kMaxL2DAttempts when the cap was hit).
template <class Real>
int grad_sample_one(const GradCell& g, int order, uint64_t seed, uint32_t cell, uint32_t t,
                    uint32_t k, Real* v, uint64_t* envelope) {
    for (int att = 0; att < kMaxL2DAttempts; ++att) {
        U4 r = draw(seed, cell, t, TAG_L2D_VEL, k, (uint32_t)(2 * att));
        U4 r2 = draw(seed, cell, t, TAG_L2D_VEL, k, (uint32_t)(2 * att + 1));
        Real n0, n1, n2, n3;
        gauss_pair<Real>(r[0], r[1], n0, n1);
        gauss_pair<Real>(r[2], r[3], n2, n3);
        const Real xi[3] = {n0, n1, n2};
        const double xd[3] = {(double)xi[0], (double)xi[1], (double)xi[2]};
        const double G = hermite_series(g.ahat, xd, order);
        const double R = u01d(r2[0]);
        if (G > g.C) *envelope += 1;
        if (g.C * R <= G) {
            for (int i = 0; i < 3; ++i) v[i] = (Real)(xd[i] + g.u[i]);
            return att + 1;
        }
    }
    for (int i = 0; i < 3; ++i) v[i] = (Real)g.u[i];
    return kMaxL2DAttempts + 1;
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
        const int64_t x = node % B.d.nx, y = node / B.d.nx;
        const int64_t cell = (y / D.p.lb_ratio) * D.p.ncx + (x / D.p.lb_ratio);
        Coeffs a;
        if (!dsmc_coefficients(&D.acc[(size_t)cell * kNumMoments], D.nsamples, D.p.ppc, a)) {
            D.status |= ST_BAD_INPUT;
            continue;
        }
        for (int q = 0; q < L.q; ++q)
            B.f[(size_t)q * B.d.nnodes + node] =
                (Real)(L.w[q] * hermite_series(a, L.xi[q].data(), B.d.order));
    }
}

template <class Real>
void map_lbm_to_dsmc(Dsmc<Real>& D, const Lbm<Real>& B, const int32_t* cells, int n) {
    const Lattice& L = B.L;
    const int r = D.p.lb_ratio;
    const uint32_t t = (uint32_t)D.step;
    std::vector<GradCell> gc(n);
    std::vector<uint32_t> nnew(n, 0);
    uint64_t total = 0;
    for (int c = 0; c < n; ++c) {
        const int64_t cell = cells[c];
        if (cell < 0 || cell >= D.d.ncells) {
            D.status |= ST_BAD_INPUT;
            return;
        }
        const int64_t ix = cell % D.p.ncx, iy = cell / D.p.ncx;
        std::vector<double> fbar(L.q, 0.0);
        for (int q = 0; q < L.q; ++q) {
            double s = 0.0;
            for (int dy = 0; dy < r; ++dy)
                for (int dx = 0; dx < r; ++dx) s += B.fa(q, ix * r + dx, iy * r + dy);
            fbar[q] = s / (double)(r * r);
        }
        gc[c] = grad_from_populations(L, fbar.data(), B.d.order);
        const double u = u01d(draw(D.p.seed, (uint32_t)cell, t, TAG_L2D_ROUND, 0, 0)[0]);
        const double ne = std::floor(gc[c].rho * (double)D.p.ppc + u);
        nnew[c] = ne > 0.0 ? (uint32_t)ne : 0u;
        total += nnew[c];
    }
    if ((int64_t)(D.ntot() + total) > D.d.capacity) {
        D.status |= ST_CAPACITY;
        return;
    }
    for (int c = 0; c < n; ++c) {
        const uint32_t cell = (uint32_t)cells[c];
        for (uint32_t i = D.cell_start[cell]; i < D.cell_start[cell + 1]; ++i) {
            if (D.x[i] >= (Real)0) D.counters[C_DELETED] += 1;
            D.x[i] = (Real)-1;
        }
    }
    for (int c = 0; c < n; ++c) {
        const uint32_t cell = (uint32_t)cells[c];
        const int ix = (int)(cell % D.p.ncx), iy = (int)(cell / D.p.ncx);
        for (uint32_t k = 0; k < nnew[c]; ++k) {
            U4 rp = draw(D.p.seed, cell, t, TAG_L2D_POS, k, 0);
            Real v[3];
            const int att = grad_sample_one<Real>(gc[c], B.d.order, D.p.seed, cell, t, k, v,
                                                  &D.counters[C_ENVELOPE]);
            if (att > kMaxL2DAttempts) {
                D.status |= ST_SAMPLING_CAP;
                D.counters[C_L2D_ATTEMPTS] += kMaxL2DAttempts;
            } else {
                D.counters[C_L2D_ATTEMPTS] += (uint64_t)att;
            }
            D.x.push_back((Real)ix + (Real)u01f(rp[0]));
            D.y.push_back((Real)iy + (Real)u01f(rp[1]));
            D.vx.push_back(v[0]);
            D.vy.push_back(v[1]);
            D.vz.push_back(v[2]);
        }
        D.counters[C_CREATED] += nnew[c];
    }
}

}  // namespace ora
