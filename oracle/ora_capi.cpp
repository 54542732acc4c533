// Oracle: C entry points for the Python test harness (ctypes).
//
// TEST INFRASTRUCTURE ONLY (see ora_common.hpp). Holds one DSMC + LBM state in host memory,
// in float or double, and exposes the steps of the method one call at a time.
#include "ora_mapping.hpp"

using namespace ora;

namespace {

struct Handle {
    int rb = 8;
    Dsmc<float> df;
    Lbm<float> lf;
    Dsmc<double> dd;
    Lbm<double> ld;
};

enum ArrayId {
    A_X = 0, A_Y = 1, A_VX = 2, A_VY = 3, A_VZ = 4, A_CELL_START = 5, A_CRMAX = 6,
    A_REM = 7, A_NBAR_SUM = 8, A_ACC = 9, A_F = 10, A_Z = 11,
};

template <class T>
int64_t copy_out(const std::vector<T>& v, void* out) {
    if (out) std::memcpy(out, v.data(), v.size() * sizeof(T));
    return (int64_t)v.size();
}
template <class T>
int set_in(std::vector<T>& v, const void* in, int64_t n, bool resize) {
    if (resize) v.resize((size_t)n);
    if ((int64_t)v.size() != n) return -1;
    std::memcpy(v.data(), in, (size_t)n * sizeof(T));
    return 0;
}

template <class Real>
int64_t get_impl(Dsmc<Real>& D, Lbm<Real>& B, int which, void* out) {
    switch (which) {
        case A_X: return copy_out(D.x, out);
        case A_Y: return copy_out(D.y, out);
        case A_VX: return copy_out(D.vx, out);
        case A_VY: return copy_out(D.vy, out);
        case A_VZ: return copy_out(D.vz, out);
        case A_CELL_START: return copy_out(D.cell_start, out);
        case A_CRMAX: return copy_out(D.crmax, out);
        case A_REM: return copy_out(D.rem, out);
        case A_NBAR_SUM: return copy_out(D.nbar_sum, out);
        case A_ACC: return copy_out(D.acc, out);
        case A_F: return copy_out(B.f, out);
        case A_Z: return copy_out(D.z, out);
    }
    return -1;
}

template <class Real>
int set_impl(Dsmc<Real>& D, Lbm<Real>& B, int which, const void* in, int64_t n) {
    switch (which) {
        case A_X: return set_in(D.x, in, n, true);
        case A_Y: return set_in(D.y, in, n, true);
        case A_VX: return set_in(D.vx, in, n, true);
        case A_VY: return set_in(D.vy, in, n, true);
        case A_VZ: return set_in(D.vz, in, n, true);
        case A_CELL_START: return set_in(D.cell_start, in, n, false);
        case A_CRMAX: return set_in(D.crmax, in, n, false);
        case A_REM: return set_in(D.rem, in, n, false);
        case A_NBAR_SUM: return set_in(D.nbar_sum, in, n, false);
        case A_ACC: return set_in(D.acc, in, n, false);
        case A_F: return set_in(B.f, in, n, false);
        case A_Z: return set_in(D.z, in, n, true);
    }
    return -1;
}

bool valid(const Params* p) {
    return p && p->ncx >= 6 && p->ncy >= 1 && (p->lb_ratio == 1 || p->lb_ratio == 2) &&
           p->ppc >= 1 && (p->lattice == 39 || p->lattice == 19) &&
           (p->real_bytes == 4 || p->real_bytes == 8) && p->sample_every >= 1 && p->kn > 0.0 &&
           p->capacity_factor >= 1.0 && std::ceil(p->capacity_factor * p->ppc) <= 256.0 &&
           (p->lb_collision == 0 || p->lb_collision == 1) && (p->d2l_mode == 0 || p->d2l_mode == 1) &&
           (p->kn_profile == 0 || (p->kn_profile == 1 && p->kn_end > 0.0)) && p->ncz >= 0 &&
           p->accum_mode == 0 && p->ncy_global >= 0 &&
           (p->ncy_global > 0 ? (p->y0 >= 0 && p->ncy >= 4 && (int64_t)p->y0 + p->ncy <= p->ncy_global)
                              : p->y0 == 0) &&
           // the channel's cells times 256 slots below 2^31 (the library's order keys)
           (double)p->ncx * (double)(p->ncy_global > 0 ? p->ncy_global : p->ncy) *
                   (double)(p->ncz >= 2 ? p->ncz : 1) * 256.0 < 2147483648.0;
}

// A streamwise slab's split move (phase_move), its outbox towards lower (dir 0) or higher
// (dir 1) rows as rows of 8 doubles (x, y, z, vx, vy, vz, tag >> 32, tag & 0xFFFFFFFF) and
// their channel cells, and the merge of the particles received from the slab below (in0) and
// above (in1) followed by the sort (phase_accept_sort).
template <class Real>
void outbox_get(Dsmc<Real>& D, int dir, double* out, uint32_t* gkey) {
    const auto& o = D.outbox[dir];
    for (size_t k = 0; k < o.size(); ++k) {
        double* r = out + 8 * k;
        r[0] = o.x[k]; r[1] = o.y[k]; r[2] = o.z[k];
        r[3] = o.vx[k]; r[4] = o.vy[k]; r[5] = o.vz[k];
        r[6] = (double)(o.tag[k] >> 32);
        r[7] = (double)(o.tag[k] & 0xFFFFFFFFull);
        gkey[k] = o.gkey[k];
    }
}
template <class Real>
void accept(Dsmc<Real>& D, const double* in[2], const uint32_t* keys[2], const int64_t n[2]) {
    typename Dsmc<Real>::Moved m[2];
    for (int b = 0; b < 2; ++b)
        for (int64_t k = 0; k < n[b]; ++k) {
            const double* r = in[b] + 8 * k;
            m[b].x.push_back((Real)r[0]); m[b].y.push_back((Real)r[1]); m[b].z.push_back((Real)r[2]);
            m[b].vx.push_back((Real)r[3]); m[b].vy.push_back((Real)r[4]); m[b].vz.push_back((Real)r[5]);
            m[b].tag.push_back(((uint64_t)r[6] << 32) | (uint64_t)r[7]);
            m[b].gkey.push_back(keys[b][k]);
        }
    D.phase_accept_sort(m, 2);
}

}  // namespace

extern "C" {

int ora_derive(const Params* p, Derived* out) {
    if (!valid(p)) return 1;
    *out = derive(*p);
    return 0;
}

void ora_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        U4 r = philox4x32_10(U4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]},
                             (uint32_t)seed, (uint32_t)(seed >> 32));
        for (int k = 0; k < 4; ++k) out[4 * i + k] = r[k];
    }
}

int ora_lattice(int q, int32_t* e, double* w, double* r) {
    if (q != 39 && q != 19) return 1;
    Lattice L = make_lattice(q);
    for (int a = 0; a < q; ++a) {
        for (int i = 0; i < 3; ++i) e[3 * a + i] = L.e[a][i];
        w[a] = L.w[a];
    }
    *r = L.r;
    return 0;
}

void* ora_create(const Params* p) {
    if (!valid(p)) return nullptr;
    Handle* h = new Handle();
    h->rb = p->real_bytes;
    if (h->rb == 4) {
        h->df.init(*p);
        h->lf.init(*p);
    } else {
        h->dd.init(*p);
        h->ld.init(*p);
    }
    return h;
}

void ora_destroy(void* hv) { delete (Handle*)hv; }

int ora_dsmc_step(void* hv, int n) {
    Handle* h = (Handle*)hv;
    for (int i = 0; i < n; ++i) (h->rb == 4) ? h->df.step_once() : h->dd.step_once();
    return 0;
}

// One phase of a DSMC step: 0 move + sort, 1 collide, 2 sample + advance the step counter.
int ora_dsmc_phase(void* hv, int phase) {
    Handle* h = (Handle*)hv;
    if (phase < 0 || phase > 2) return 1;
    if (h->rb == 4) {
        if (phase == 0) h->df.phase_move_sort();
        if (phase == 1) h->df.phase_collide();
        if (phase == 2) h->df.phase_sample_advance();
    } else {
        if (phase == 0) h->dd.phase_move_sort();
        if (phase == 1) h->dd.phase_collide();
        if (phase == 2) h->dd.phase_sample_advance();
    }
    return 0;
}

// A streamwise slab's split move, its outboxes and the merge of what it received.
void ora_dsmc_move(void* hv) {
    Handle* h = (Handle*)hv;
    (h->rb == 4) ? h->df.phase_move() : h->dd.phase_move();
}

int64_t ora_outbox_size(void* hv, int dir) {
    Handle* h = (Handle*)hv;
    return (int64_t)((h->rb == 4) ? h->df.outbox[dir & 1].size() : h->dd.outbox[dir & 1].size());
}

void ora_outbox_get(void* hv, int dir, double* out, uint32_t* gkey) {
    Handle* h = (Handle*)hv;
    if (h->rb == 4) outbox_get(h->df, dir & 1, out, gkey);
    else outbox_get(h->dd, dir & 1, out, gkey);
}

void ora_dsmc_accept(void* hv, const double* in0, const uint32_t* k0, int64_t n0, const double* in1,
                     const uint32_t* k1, int64_t n1) {
    Handle* h = (Handle*)hv;
    const double* in[2] = {in0, in1};
    const uint32_t* keys[2] = {k0, k1};
    const int64_t n[2] = {n0, n1};
    if (h->rb == 4) accept(h->df, in, keys, n);
    else accept(h->dd, in, keys, n);
}

int ora_lbm_step(void* hv, int n) {
    Handle* h = (Handle*)hv;
    for (int i = 0; i < n; ++i) (h->rb == 4) ? h->lf.step_once() : h->ld.step_once();
    return 0;
}

int ora_map_dsmc_to_lbm(void* hv, const int32_t* nodes, int n) {
    Handle* h = (Handle*)hv;
    if (h->rb == 4) map_dsmc_to_lbm(h->df, h->lf, nodes, n);
    else map_dsmc_to_lbm(h->dd, h->ld, nodes, n);
    return 0;
}

int ora_map_lbm_to_dsmc(void* hv, const int32_t* cells, int n) {
    Handle* h = (Handle*)hv;
    if (h->rb == 4) map_lbm_to_dsmc(h->df, h->lf, cells, n);
    else map_lbm_to_dsmc(h->dd, h->ld, cells, n);
    return 0;
}

int64_t ora_get(void* hv, int which, void* out) {
    Handle* h = (Handle*)hv;
    return (h->rb == 4) ? get_impl(h->df, h->lf, which, out) : get_impl(h->dd, h->ld, which, out);
}

int ora_set(void* hv, int which, const void* in, int64_t n) {
    Handle* h = (Handle*)hv;
    return (h->rb == 4) ? set_impl(h->df, h->lf, which, in, n) : set_impl(h->dd, h->ld, which, in, n);
}

// scalars: [0] step, [1] nsamples, [2] status, [3] ntot
void ora_scalars(void* hv, uint64_t* out) {
    Handle* h = (Handle*)hv;
    if (h->rb == 4) {
        out[0] = h->df.step; out[1] = h->df.nsamples; out[2] = h->df.status; out[3] = h->df.ntot();
    } else {
        out[0] = h->dd.step; out[1] = h->dd.nsamples; out[2] = h->dd.status; out[3] = h->dd.ntot();
    }
}

void ora_set_scalars(void* hv, uint64_t step, uint64_t nsamples) {
    Handle* h = (Handle*)hv;
    if (h->rb == 4) { h->df.step = step; h->df.nsamples = nsamples; }
    else { h->dd.step = step; h->dd.nsamples = nsamples; }
}

void ora_counters(void* hv, uint64_t* out) {
    Handle* h = (Handle*)hv;
    const uint64_t* c = (h->rb == 4) ? h->df.counters : h->dd.counters;
    for (int i = 0; i < C_NUM; ++i) out[i] = c[i];
}

// Per-node g_y and tau for the LBM of the handle (n = nnodes), or none (n = 0).
// The Kn profile of the configuration p at its own rows: the NTC factors of DSMC cell rows
// [crow0, crow0 + ncrows) and tau of LB rows [nrow0, nrow0 + nnrows) (either count may be 0).
int ora_kn_profile_rows(const Params* p, int64_t crow0, int64_t ncrows, double* coll,
                        int64_t nrow0, int64_t nnrows, double* tau) {
    const Derived d = derive(*p);
    for (int64_t i = 0; i < ncrows; ++i) coll[i] = kn_cell_coll(*p, d, crow0 + i);
    for (int64_t i = 0; i < nnrows; ++i) tau[i] = kn_node_tau(*p, d, nrow0 + i);
    return 0;
}

// Per-cell NTC factors (n = ncells), or the scalar factor again (n = 0).
int ora_dsmc_cell_coll(void* hv, const double* coll, int64_t n) {
    Handle* h = (Handle*)hv;
    auto set = [&](auto& D) {
        if (n == 0) {
            D.coll_cell.clear();
            return 0;
        }
        if (n != D.d.ncells) return 1;
        D.coll_cell.assign(coll, coll + n);
        return 0;
    };
    return (h->rb == 4) ? set(h->df) : set(h->dd);
}

int ora_lbm_node_params(void* hv, const double* g, const double* tau, int64_t n) {
    Handle* h = (Handle*)hv;
    auto set = [&](auto& B) {
        if (n == 0) {
            B.g_node.clear();
            B.tau_node.clear();
            return 0;
        }
        if (n != B.d.nnodes) return 1;
        B.g_node.assign(g, g + n);
        B.tau_node.assign(tau, tau + n);
        return 0;
    };
    return (h->rb == 4) ? set(h->lf) : set(h->ld);
}

// Grad coefficients of one node's populations (20 values) and the interface loss over the
// listed nodes against 20 targets per node.
int ora_lbm_grad_node(void* hv, int64_t node, double* out) {
    Handle* h = (Handle*)hv;
    if (h->rb == 4) h->lf.grad_node(node, out);
    else h->ld.grad_node(node, out);
    return 0;
}
double ora_lbm_interface_loss(void* hv, const int32_t* nodes, int n, const double* targets) {
    Handle* h = (Handle*)hv;
    return (h->rb == 4) ? h->lf.interface_loss(nodes, n, targets)
                        : h->ld.interface_loss(nodes, n, targets);
}

// One node's collision from streamed populations fs (double), for pins.
int ora_lbm_collide(const Params* p, const double* fs, double* out) {
    if (!valid(p)) return 1;
    Lbm<double> B;
    B.p = *p;
    B.d = derive(*p);
    B.L = make_lattice(p->lattice);
    B.collide(fs, out);
    return 0;
}

// DSMC2LB populations of one node from 20 cumulative sums over S samples.
int ora_dsmc2lb_node(int q, const double* m, uint64_t S, int ppc, double* out) {
    if (q != 39 && q != 19) return 1;
    Lattice L = make_lattice(q);
    Coeffs a;
    if (!dsmc_coefficients(m, S, ppc, a)) return 2;
    for (int k = 0; k < q; ++k) out[k] = L.w[k] * hermite_series(a, L.xi[k].data(), q == 39 ? 3 : 2);
    return 0;
}

// The float series of ln, sin and cos used by the float state path (for their pins).
void ora_float_funcs(const float* x, int64_t n, float* ln_out, float* sin_out, float* cos_out) {
    for (int64_t i = 0; i < n; ++i) {
        if (ln_out) ln_out[i] = ln_f(x[i]);
        if (sin_out || cos_out) {
            float s, c;
            sincos2pi_f(x[i], s, c);
            if (sin_out) sin_out[i] = s;
            if (cos_out) cos_out[i] = c;
        }
    }
}

// Gaussian pairs in the state precision from Philox words (for the float-path pins).
void ora_gauss_pairs(const uint32_t* r, int64_t n, int real_bytes, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        if (real_bytes == 4) {
            float a, b;
            gauss_pair<float>(r[2 * i], r[2 * i + 1], a, b);
            out[2 * i] = a;
            out[2 * i + 1] = b;
        } else {
            gauss_pair<double>(r[2 * i], r[2 * i + 1], out[2 * i], out[2 * i + 1]);
        }
    }
}

// Grad coefficients of a population vector: out = [rho, u(3), a2(9), a3(27), M, C].
int ora_grad_coeffs(int q, const double* f, double* out) {
    if (q != 39 && q != 19) return 1;
    Lattice L = make_lattice(q);
    GradCell g = grad_from_populations(L, f, q == 39 ? 3 : 2);
    out[0] = g.rho;
    for (int i = 0; i < 3; ++i) out[1 + i] = g.u[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            out[4 + 3 * i + j] = g.ahat.a2[i][j];
            for (int k = 0; k < 3; ++k) out[13 + 9 * i + 3 * j + k] = g.ahat.a3[i][j][k];
        }
    out[40] = g.M;
    out[41] = g.C;
    return 0;
}

// The FP64 coefficients packed by symmetry and rounded to the precision real_bytes, as the
// sampler uses them: out = [rho, u(3), a2(6), a3(10), M, C] (packed order; rho and M in FP64).
int ora_grad_coeffs_packed(int q, const double* f, int real_bytes, double* out) {
    if (q != 39 && q != 19) return 1;
    Lattice L = make_lattice(q);
    const int order = q == 39 ? 3 : 2;
    const GradCell g = grad_from_populations(L, f, order);
    auto put = [&](const auto& p) {
        out[0] = g.rho;
        for (int i = 0; i < 3; ++i) out[1 + i] = p.u[i];
        for (int k = 0; k < 6; ++k) out[4 + k] = p.a2[k];
        for (int k = 0; k < 10; ++k) out[10 + k] = p.a3[k];
        out[20] = g.M;
        out[21] = p.C;
    };
    if (real_bytes == 4)
        put(pack<float>(g));
    else
        put(pack<double>(g));
    return 0;
}

// Table 1 sampler: nsamp particles of one cell from one population vector, in double.
// info = [trials, envelope violations, capped].
int ora_grad_sample(int q, const double* f, uint64_t seed, uint32_t cell, uint32_t t,
                    int64_t nsamp, double* v_out, uint64_t* info) {
    if (q != 39 && q != 19) return 1;
    if (nsamp > 4000000) return 2;
    Lattice L = make_lattice(q);
    const int order = q == 39 ? 3 : 2;
    GradCell g = grad_from_populations(L, f, order);
    std::vector<double> out(6 * (size_t)nsamp);
    uint64_t env = 0;
    bool capped = false;
    const uint64_t trials = grad_sample_cell<double>(pack<double>(g), order, seed, cell, t,
                                                     (uint32_t)nsamp, 0.0, 0.0, 0.0, false, out.data(),
                                                     &env, &capped);
    for (int64_t k = 0; k < nsamp; ++k)
        for (int i = 0; i < 3; ++i) v_out[3 * k + i] = out[6 * k + 3 + i];
    info[0] = trials;
    info[1] = env;
    info[2] = capped ? 1 : 0;
    return 0;
}

// G in the state precision (packed grouping) and in double (full tensors), for its pin.
int ora_grad_G(int q, const double* f, const double* xi, int64_t n, int real_bytes, double* out) {
    if (q != 39 && q != 19) return 1;
    Lattice L = make_lattice(q);
    const int order = q == 39 ? 3 : 2;
    GradCell g = grad_from_populations(L, f, order);
    for (int64_t k = 0; k < n; ++k) {
        if (real_bytes == 4) {
            GradPacked<float> p = pack<float>(g);
            const float x[3] = {(float)xi[3 * k], (float)xi[3 * k + 1], (float)xi[3 * k + 2]};
            out[2 * k] = grad_G<float>(p.a2, p.a3, x, order);
        } else {
            GradPacked<double> p = pack<double>(g);
            out[2 * k] = grad_G<double>(p.a2, p.a3, &xi[3 * k], order);
        }
        out[2 * k + 1] = hermite_series(g.ahat, &xi[3 * k], order);
    }
    return 0;
}

}  // extern "C"
