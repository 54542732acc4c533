// Oracle: regularised lattice-Boltzmann stream-collide with diffuse kinetic walls and a
// body force, on D3Q39 (Hermite order 3) or D3Q19 (order 2).
//
// TEST INFRASTRUCTURE ONLY (see ora_common.hpp). Every node is updated with double
// arithmetic by full-tensor loops over the Hermite expansion of Sec. 2 (Eq. series,
// Eq. coefficients_LBM), so each step can be read against its definition:
//   pull streaming along e_a; populations entering through a wall are re-emitted by the
//   wall Maxwellian at rest with the wall density that balances the mass leaving through
//   that wall on the same streamwise row (the "kinetic boundary conditions" of Sec. 2);
//   rho = sum f, rho u = sum f xi + rho g / 2;
//   f_eq = w rho sum_{n<=N} u^n : H^n / n!;
//   f_neq projected onto H1, H2 (and H3) by the quadrature (the "regularization" of
//   Sec. 2);
//   F = w sum_{n=1..N} n (g (x) a_eq^(n-1)) : H^n / n! (Hermite expansion of -g . grad_xi f);
//   f' = f_eq + (1 - 1/tau) f_neq_reg + (1 - 1/(2 tau)) F,
// or, with lb_collision = 1 (the unregularised LB of the proof-of-concept hybrid, Sec. 4),
//   f' = f_eq + (1 - 1/tau) (f - f_eq) + (1 - 1/(2 tau)) F.
// Relaxation time from Eq. tau. The quasi-2D slab has one periodic layer in z.
//
// Optional per-node parameters (for the differentiated LBM): a body-force increment g_y and
// a relaxation time tau for every node; when set they replace the scalars of Eq. tau and of
// the force. The coupling-interface loss of the differentiated LBM is defined here too: at
// each listed node, the Grad coefficients of its populations (rho, u = sum f xi / rho,
// a2 = sum f c c / rho - I, a3 = sum f c c c / rho with c = xi - u; the comoving coefficients
// of Table 1) against 20 target values, summed as squares.
#pragma once
#include "ora_common.hpp"

namespace ora {

template <class Real>
struct Lbm {
    Params p;
    Derived d;
    Lattice L;
    std::vector<Real> f;  // f[a * nnodes + y * nx + x]
    std::vector<double> g_node, tau_node;  // per-node g_y and tau; empty: the scalars

    void init(const Params& pp) {
        p = pp;
        d = derive(p);
        L = make_lattice(p.lattice);
        f.assign((size_t)L.q * d.nnodes, 0);
        for (int a = 0; a < L.q; ++a)
            for (int64_t n = 0; n < d.nnodes; ++n) f[(size_t)a * d.nnodes + n] = (Real)L.w[a];
        g_node.clear();
        tau_node.clear();
        if (p.kn_profile == 1) {  // tau of Eq. tau at each node's Kn, the force of kn
            g_node.assign((size_t)d.nnodes, d.g_step);
            tau_node.resize((size_t)d.nnodes);
            for (int64_t n = 0; n < d.nnodes; ++n)
                tau_node[(size_t)n] = kn_node_tau(p, d, channel_lb_row(p, d, (n / d.nx) % d.ny));
        }
    }

    double fa(int a, int64_t x, int64_t y, int64_t z = 0) const {
        return (double)f[(size_t)a * d.nnodes + (z * d.ny + y) * d.nx + x];
    }
    int64_t wrap_y(int64_t y) const { return ((y % d.ny) + d.ny) % d.ny; }
    int64_t wrap_z(int64_t z) const { return ((z % d.nz) + d.nz) % d.nz; }

    // Collision of one node given its streamed populations fs[q]; writes out[q].
    void collide(const double* fs, double* out) const { collide(fs, out, d.g_step, d.tau); }
    void collide(const double* fs, double* out, double gy, double tau) const {
        const int N = d.order;
        double rho = 0.0, j[3] = {0, 0, 0};
        for (int a = 0; a < L.q; ++a) {
            rho += fs[a];
            for (int i = 0; i < 3; ++i) j[i] += fs[a] * L.xi[a][i];
        }
        const double g[3] = {0.0, gy, 0.0};
        double u[3];
        for (int i = 0; i < 3; ++i) u[i] = (j[i] + 0.5 * rho * g[i]) / rho;

        Coeffs aeq{};
        aeq.a0 = rho;
        for (int i = 0; i < 3; ++i) {
            aeq.a1[i] = rho * u[i];
            for (int k = 0; k < 3; ++k) {
                aeq.a2[i][k] = rho * u[i] * u[k];
                for (int l = 0; l < 3; ++l) aeq.a3[i][k][l] = rho * u[i] * u[k] * u[l];
            }
        }
        std::vector<double> feq(L.q), fneq(L.q);
        for (int a = 0; a < L.q; ++a) {
            feq[a] = L.w[a] * hermite_series(aeq, L.xi[a].data(), N);
            fneq[a] = fs[a] - feq[a];
        }
        // Projection of f_neq onto H1..HN. The H1 part is -rho g / 2 (the half-step force
        // shift of u); keeping it makes the momentum gained per step exactly rho g.
        Coeffs aneq = project(L, fneq.data());
        aneq.a0 = 0.0;
        if (N < 3) std::memset(aneq.a3, 0, sizeof(aneq.a3));

        Coeffs bf{};
        for (int i = 0; i < 3; ++i) {
            bf.a1[i] = g[i] * aeq.a0;
            for (int k = 0; k < 3; ++k) {
                bf.a2[i][k] = 2.0 * g[i] * aeq.a1[k];
                for (int l = 0; l < 3; ++l) bf.a3[i][k][l] = 3.0 * g[i] * aeq.a2[k][l];
            }
        }
        const double om = 1.0 - 1.0 / tau;
        const double of = 1.0 - 1.0 / (2.0 * tau);
        for (int a = 0; a < L.q; ++a) {
            const double* x = L.xi[a].data();
            const double freg = p.lb_collision == 1 ? fneq[a] : L.w[a] * hermite_series(aneq, x, N);
            const double F = L.w[a] * hermite_series(bf, x, N);
            out[a] = feq[a] + om * freg + of * F;
        }
    }

    void step_once() {
        const int64_t nx = d.nx, ny = d.ny;
        std::vector<Real> nf(f.size());
        // Mass flux normalisation of the wall Maxwellian: sum over incoming a of e_x w_a.
        double flux_norm = 0.0;
        for (int a = 0; a < L.q; ++a)
            if (L.e[a][0] > 0) flux_norm += L.e[a][0] * L.w[a];
        // wall densities of every streamwise row (y, z); in 3D the pull is periodic in z too
        const int64_t nz = d.nz;
        std::vector<double> rhoL(ny * nz), rhoR(ny * nz);
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y) {
                double ml = 0.0, mr = 0.0;
                for (int a = 0; a < L.q; ++a) {
                    const int ex = L.e[a][0];
                    const int64_t sy = wrap_y(y - L.e[a][1]);
                    const int64_t sz = wrap_z(z - L.e[a][2]);
                    if (ex < 0)
                        for (int64_t i = 0; i < -ex; ++i) ml += fa(a, i, sy, sz);
                    if (ex > 0)
                        for (int64_t i = nx - ex; i < nx; ++i) mr += fa(a, i, sy, sz);
                }
                rhoL[z * ny + y] = ml / flux_norm;
                rhoR[z * ny + y] = mr / flux_norm;
            }
        std::vector<double> fs(L.q), out(L.q);
        for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                for (int a = 0; a < L.q; ++a) {
                    const int64_t sx = x - L.e[a][0];
                    const int64_t sy = wrap_y(y - L.e[a][1]);
                    const int64_t sz = wrap_z(z - L.e[a][2]);
                    if (sx < 0)
                        fs[a] = L.w[a] * rhoL[z * ny + y];
                    else if (sx >= nx)
                        fs[a] = L.w[a] * rhoR[z * ny + y];
                    else
                        fs[a] = fa(a, sx, sy, sz);
                }
                const int64_t node = (z * ny + y) * nx + x;
                if (g_node.empty())
                    collide(fs.data(), out.data());
                else
                    collide(fs.data(), out.data(), g_node[(size_t)node], tau_node[(size_t)node]);
                for (int a = 0; a < L.q; ++a) nf[(size_t)a * d.nnodes + node] = (Real)out[a];
            }
        f.swap(nf);
    }

    // Grad coefficients of the populations of one node, by their definitions: out[0] rho,
    // out[1..3] u, out[4..9] a2 (xx xy xz yy yz zz), out[10..19] a3 (xxx xxy xxz xyy xyz
    // xzz yyy yyz yzz zzz).
    void grad_node(int64_t node, double* out) const {
        double rho = 0.0, j[3] = {0, 0, 0};
        for (int a = 0; a < L.q; ++a) {
            const double fa_ = (double)f[(size_t)a * d.nnodes + node];
            rho += fa_;
            for (int i = 0; i < 3; ++i) j[i] += fa_ * L.xi[a][i];
        }
        double u[3];
        for (int i = 0; i < 3; ++i) u[i] = j[i] / rho;
        double m2[3][3] = {}, m3[3][3][3] = {};
        for (int a = 0; a < L.q; ++a) {
            const double fa_ = (double)f[(size_t)a * d.nnodes + node];
            double c[3];
            for (int i = 0; i < 3; ++i) c[i] = L.xi[a][i] - u[i];
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) {
                    m2[i][k] += fa_ * c[i] * c[k];
                    for (int l = 0; l < 3; ++l) m3[i][k][l] += fa_ * c[i] * c[k] * c[l];
                }
        }
        out[0] = rho;
        for (int i = 0; i < 3; ++i) out[1 + i] = u[i];
        const int p2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        for (int k = 0; k < 6; ++k) {
            const int i = p2[k][0], l = p2[k][1];
            out[4 + k] = m2[i][l] / rho - (i == l ? 1.0 : 0.0);
        }
        const int p3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                               {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
        for (int k = 0; k < 10; ++k) out[10 + k] = m3[p3[k][0]][p3[k][1]][p3[k][2]] / rho;
    }

    // Coupling-interface loss: sum over the listed nodes of the squared differences between
    // their 20 Grad coefficients and the targets (20 per node).
    double interface_loss(const int32_t* nodes, int n, const double* targets) const {
        double loss = 0.0;
        for (int k = 0; k < n; ++k) {
            double m[20];
            grad_node(nodes[k], m);
            for (int i = 0; i < 20; ++i) {
                const double e = m[i] - targets[20 * k + i];
                loss += e * e;
            }
        }
        return loss;
    }
};

}  // namespace ora
