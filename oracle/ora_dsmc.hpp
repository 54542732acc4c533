// Oracle: DSMC particle step (move with diffuse isothermal walls, cell sort, NTC hard-sphere
// collisions, per-cell Hermite-moment sampling).
//
// TEST INFRASTRUCTURE ONLY (see ora_common.hpp). Plain loops in the order Bird's DSMC step
// takes them (move -> index -> collide -> sample), which the paper adopts in Sec. 5
// (Eq. collisionnumber and the NTC scheme it names). With Real = float the arithmetic is the
// float arithmetic the GPU state uses, step for step, so that cell keys, the sort
// permutation and the selected collision pairs can be compared bit for bit; the random
// normals and wall speeds use the float series of ora_common.hpp in that mode.
#pragma once
#include <algorithm>
#include <cstring>
#include <numeric>

#include "ora_common.hpp"

namespace ora {

constexpr int kMaxBounces = 8;        // wall interactions per particle per step
constexpr int kMaxScatterBlocks = 16; // Marsaglia attempts = 2 per block
constexpr uint32_t kDeadKey = 0xFFFFFFFFu;
constexpr int kNumMoments = 20;

enum Counter {
    C_WALL_HITS = 0,
    C_CANDIDATES = 1,
    C_COLLISIONS = 2,
    C_CREATED = 3,
    C_DELETED = 4,
    C_L2D_ATTEMPTS = 5,
    C_ENVELOPE = 6,
    C_BOUNCE_CAP = 7,
    C_NUM = 16,
};

template <class Real>
struct Dsmc {
    Params p;
    Derived d;
    // Particle state, ordered by cell after every step (Sec. 5, "per cell" NTC).
    std::vector<Real> x, y, vx, vy, vz;
    std::vector<Real> z;  // 3D only (ncz >= 2), else empty
    std::vector<uint32_t> cell_start;  // ncells + 1
    // Per-cell collision state of the NTC scheme.
    std::vector<Real> crmax;           // (sigma_T c_r)_max / sigma_T
    std::vector<Real> rem;             // fractional candidate carried to the next step
    std::vector<double> coll_cell;     // per-cell NTC factor (kn_profile = 1), else empty
    std::vector<uint32_t> nbar_sum;    // sum of N over steps, for N-bar = <N>
    // Cumulative sums for the DSMC2LB mapping (Sec. 2.1 "cumulative averages"):
    // [N, S vx, vy, vz, S vv (xx xy xz yy yz zz), S vvv (xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz)]
    std::vector<double> acc;
    uint64_t step = 0, nsamples = 0;
    uint32_t status = 0;
    uint64_t counters[C_NUM] = {};

    void init(const Params& pp) {
        p = pp;
        d = derive(p);
        const int64_t n = d.ncells * p.ppc;
        x.assign(n, 0); y.assign(n, 0); vx.assign(n, 0); vy.assign(n, 0); vz.assign(n, 0);
        z.assign(three_d() ? n : 0, 0);
        cell_start.assign(d.ncells + 1, 0);
        // Sec. 3.1: a fixed number of particles placed in each cell, Maxwellian at T
        // (Eq. globalMax with unit variance), drawn by Box-Muller.
        for (int64_t c = 0; c < d.ncells; ++c) {
            // the channel's row and cell id (a streamwise slab holds rows y0 .. y0 + ncy - 1)
            const int ix = (int)(c % p.ncx), iy = y0() + (int)((c / p.ncx) % p.ncy);
            const int iz = (int)(c / ((int64_t)p.ncx * p.ncy));
            const uint32_t gc = channel_cell(p, c);
            cell_start[c] = (uint32_t)(c * p.ppc);
            for (int k = 0; k < p.ppc; ++k) {
                const int64_t s = c * p.ppc + k;
                U4 rp = draw(p.seed, gc, 0, TAG_INIT_POS, (uint32_t)k, 0);
                x[s] = (Real)ix + (Real)u01f(rp[0]);
                y[s] = (Real)iy + (Real)u01f(rp[1]);
                if (three_d()) z[s] = (Real)iz + (Real)u01f(rp[2]);
                U4 rv = draw(p.seed, gc, 0, TAG_INIT_VEL, (uint32_t)k, 0);
                Real n0, n1, n2, n3;
                gauss_pair<Real>(rv[0], rv[1], n0, n1);
                gauss_pair<Real>(rv[2], rv[3], n2, n3);
                vx[s] = n0;
                vy[s] = n1;
                vz[s] = n2;
            }
        }
        cell_start[d.ncells] = (uint32_t)n;
        crmax.assign(d.ncells, (Real)p.crmax_init);
        rem.assign(d.ncells, (Real)0);
        coll_cell.clear();
        if (p.kn_profile == 1) {  // Eq. collisionnumber at each cell centre's Kn
            coll_cell.resize((size_t)d.ncells);
            for (int64_t c = 0; c < d.ncells; ++c)
                coll_cell[(size_t)c] = kn_cell_coll(p, d, y0() + (c / p.ncx) % p.ncy);
        }
        nbar_sum.assign(d.ncells, 0u);
        acc.assign(d.ncells * kNumMoments, 0.0);
        step = 0;
        nsamples = 0;
        status = 0;
        std::memset(counters, 0, sizeof(counters));
    }

    size_t ntot() const { return x.size(); }
    bool three_d() const { return p.ncz >= 2; }
    int y0() const { return p.ncy_global > 0 ? p.y0 : 0; }

    // Particles that left a streamwise slab in the last move, towards lower (0) and higher
    // (1) rows of the channel, with their order tags (order_tag) and new channel cells; and
    // the particles received from the neighbours.
    struct Moved {
        std::vector<Real> x, y, z, vx, vy, vz;
        std::vector<uint64_t> tag;
        std::vector<uint32_t> gkey;
        void clear() {
            x.clear(); y.clear(); z.clear(); vx.clear(); vy.clear(); vz.clear();
            tag.clear(); gkey.clear();
        }
        size_t size() const { return x.size(); }
    };
    Moved outbox[2];
    std::vector<uint32_t> key_;   // new local cell of each particle after the move
    std::vector<uint64_t> tag_;   // order tag of each particle (order_tag)

    // Diffuse isothermal re-emission from a wall at rest (Sec. 3.1, "fully diffuse
    // reflection"): normal speed from the flux-weighted Maxwellian sqrt(-2 ln U), tangential
    // components Gaussian. `sign` points into the gas. Draws are keyed by the particle's cell
    // and rank in that cell at the start of the step, and the bounce number.
    void reemit(uint32_t cell, uint32_t rank, uint32_t s, int bounce, Real sign, Real& ux, Real& uy,
                Real& uz) {
        U4 r = draw(p.seed, cell, s, TAG_WALL, (rank << 3) | (uint32_t)bounce, 0);
        const Real vn = wall_speed<Real>(r[0]);
        Real t1, t2;
        gauss_pair<Real>(r[1], r[2], t1, t2);
        ux = sign * vn;
        uy = t1;
        uz = t2;
    }

    // The channel's cell (iz rows + iy) ncx + ix of a position.
    uint32_t cell_key(Real xx, Real yy, Real zz) const {
        const int rows = (int)channel_rows(p);
        int ix = (int)std::floor(xx);
        int iy = (int)std::floor(yy);
        if (ix < 0) ix = 0;
        if (ix > p.ncx - 1) ix = p.ncx - 1;
        if (iy < 0) iy = 0;
        if (iy > rows - 1) iy = rows - 1;
        int iz = 0;
        if (three_d()) {
            iz = (int)std::floor(zz);
            if (iz < 0) iz = 0;
            if (iz > p.ncz - 1) iz = p.ncz - 1;
        }
        return (uint32_t)(((int64_t)iz * rows + iy) * p.ncx + ix);
    }

    // The slab's own cell of a channel cell, or -1 (with the direction to the neighbour that
    // holds it: 0 lower rows, 1 higher rows, the nearer way around the periodic channel).
    int64_t local_cell(uint32_t gk, int& dir) const {
        const int64_t rows = channel_rows(p);
        const int64_t plane = (int64_t)p.ncx * rows;
        const int64_t iz = gk / plane, r = gk % plane, iy = r / p.ncx, ix = r % p.ncx;
        const int64_t iyl = iy - y0();
        if (iyl >= 0 && iyl < p.ncy) {
            dir = -1;
            return (iz * p.ncy + iyl) * p.ncx + ix;
        }
        const int64_t above = ((iy - (y0() + p.ncy)) % rows + rows) % rows;
        const int64_t below = ((y0() - 1 - iy) % rows + rows) % rows;
        dir = above <= below ? 1 : 0;
        return -1;
    }

    // Periodic wrap of a coordinate into [0, period).
    static Real wrap(Real v, Real period) {
        if (v < (Real)0 || v >= period) {
            v = v - period * std::floor(v / period);
            if (v < (Real)0) v = v + period;
            if (v >= period) v = v - period;
        }
        return v;
    }

    // Move one particle through one time step: body-force kick, free flight, wall hits,
    // periodic wrap in the streamwise direction. `cell` is the particle's channel cell (the
    // key of its wall draws). Returns the new channel cell.
    uint32_t move_one(uint32_t i, uint32_t s, uint32_t cell, uint32_t rank) {
        if (!(x[i] >= (Real)0)) return kDeadKey;  // deleted by a coupling step
        const Real H = (Real)p.ncx;
        const Real L = (Real)channel_rows(p);
        const bool td = three_d();
        Real px = x[i], py = y[i], pz = td ? z[i] : (Real)0;
        Real ux = vx[i], uy = vy[i] + (Real)d.g_step, uz = vz[i];
        Real t = (Real)d.dt;
        for (int b = 0;; ++b) {
            const Real xn = px + ux * t;
            const bool left = xn < (Real)0;
            const bool right = xn > H;
            if (!left && !right) {
                px = xn;
                py = py + uy * t;
                if (td) pz = pz + uz * t;
                break;
            }
            if (b == kMaxBounces) {
                status |= ST_BOUNCE_CAP;
                counters[C_BOUNCE_CAP] += 1;
                px = left ? (Real)0 : H;
                py = py + uy * t;
                if (td) pz = pz + uz * t;
                break;
            }
            counters[C_WALL_HITS] += 1;
            Real th = left ? px / (-ux) : (H - px) / ux;
            py = py + uy * th;
            if (td) pz = pz + uz * th;
            px = left ? (Real)0 : H;
            t = t - th;
            if (t < (Real)0) t = (Real)0;
            reemit(cell, rank, s, b, left ? (Real)1 : (Real)-1, ux, uy, uz);
        }
        py = wrap(py, L);
        if (td) pz = wrap(pz, (Real)p.ncz);
        x[i] = px;
        y[i] = py;
        if (td) z[i] = pz;
        vx[i] = ux;
        vy[i] = uy;
        vz[i] = uz;
        return cell_key(px, py, pz);
    }

    // The order of the particles of a cell before its collide (the paper does not fix one): a
    // particle that came from a cell at most one cell away along every axis comes first,
    // ordered by the offset o = 3 (dy + 1) + dx + 1 in 2D, 9 (dz + 1) + 3 (dy + 1) + dx + 1
    // in 3D, of its displacement (dx, dy, dz) from its old cell to its new one, then by its
    // rank in its old cell. The streamwise and spanwise displacements are periodic; where
    // +1 and -1 are the same cell (a period of two), it counts as +1. Every other particle
    // follows, ordered by its old channel cell, then rank. Returns the particle's tag, which
    // sorts in this order.
    uint64_t order_tag(uint32_t g_old, uint32_t g_new, uint32_t rank) const {
        const int64_t nx = p.ncx, ny = channel_rows(p);
        const int64_t ox = g_old % nx, oy = (g_old / nx) % ny, oz = g_old / (nx * ny);
        const int64_t mx = g_new % nx, my = (g_new / nx) % ny, mz = g_new / (nx * ny);
        auto periodic = [](int64_t d, int64_t period) -> int {  // -1, 0, 1, or 2: farther
            const int64_t e = ((d % period) + period) % period;
            if (e == 0) return 0;
            if (e == 1) return 1;
            if (e == period - 1) return -1;
            return 2;
        };
        const int64_t dx = mx - ox;
        const int dy = periodic(my - oy, ny);
        const int dz = three_d() ? periodic(mz - oz, p.ncz) : 0;
        if (dx < -1 || dx > 1 || dy == 2 || dz == 2)
            return (1ull << 63) | ((uint64_t)g_old << 32) | rank;
        const uint64_t o = three_d() ? (uint64_t)(9 * (dz + 1) + 3 * (dy + 1) + (dx + 1))
                                     : (uint64_t)(3 * (dy + 1) + (dx + 1));
        return (o << 32) | rank;
    }

    // Order by cell key; within a cell by the particles' tags (order_tag), the received
    // particles of a streamwise slab merged in. Deleted particles are dropped.
    void sort_by_cell(const std::vector<uint32_t>& key, const std::vector<uint64_t>& tag) {
        std::vector<uint32_t> idx;
        idx.reserve(key.size());
        for (uint32_t i = 0; i < key.size(); ++i)
            if (key[i] != kDeadKey) idx.push_back(i);
        std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
            return key[a] < key[b] || (key[a] == key[b] && tag[a] < tag[b]);
        });
        auto permute = [&](std::vector<Real>& v) {
            std::vector<Real> o(idx.size());
            for (size_t k = 0; k < idx.size(); ++k) o[k] = v[idx[k]];
            v.swap(o);
        };
        permute(x); permute(y); permute(vx); permute(vy); permute(vz);
        if (three_d()) permute(z);
        std::fill(cell_start.begin(), cell_start.end(), 0u);
        for (uint32_t i : idx) cell_start[key[i] + 1] += 1;
        for (int64_t c = 0; c < d.ncells; ++c) {
            if (cell_start[c + 1] > (uint32_t)d.bin) status |= ST_CAPACITY;  // bin overflow
            cell_start[c + 1] += cell_start[c];
        }
    }

    // Isotropic unit vector by Marsaglia (1972): (u1, u2) uniform in the unit disc,
    // n = (2 u1 sqrt(1-s), 2 u2 sqrt(1-s), 1 - 2 s).
    bool unit_vector(uint32_t c, uint32_t s, uint32_t k, Real* n) {
        for (int blk = 0; blk < kMaxScatterBlocks; ++blk) {
            U4 r = draw(p.seed, c, s, TAG_NTC_SCAT, k, (uint32_t)blk);
            for (int h = 0; h < 2; ++h) {
                const Real u1 = (Real)2 * (Real)u01f(r[2 * h]) - (Real)1;
                const Real u2 = (Real)2 * (Real)u01f(r[2 * h + 1]) - (Real)1;
                const Real ss = u1 * u1 + u2 * u2;
                if (ss < (Real)1) {
                    const Real a = (Real)2 * std::sqrt((Real)1 - ss);
                    n[0] = u1 * a;
                    n[1] = u2 * a;
                    n[2] = (Real)1 - (Real)2 * ss;
                    return true;
                }
            }
        }
        return false;
    }

    // NTC hard-sphere collisions in one cell (Sec. 5, Eq. collisionnumber):
    // N_cand = 1/2 N Nbar F_N (sigma_T c_r)_max dt / V_c plus the carried remainder; each
    // candidate pair (i, j != i) collides with probability c_r / c_r,max; post-collision
    // velocities are v_cm +- c_r n / 2 with n isotropic (hard spheres).
    void collide_cell(uint32_t c, uint32_t s) {
        const uint32_t gc = channel_cell(p, c);  // the key of the cell's random streams
        const uint32_t base = cell_start[c];
        const uint32_t n = cell_start[c + 1] - base;
        nbar_sum[c] += n;
        const Real nbar = (Real)nbar_sum[c] / (Real)(s + 1);
        if (n < 2) return;
        const Real cdt = (Real)(coll_cell.empty() ? d.coll_dt : coll_cell[c]);
        const Real ncand = (Real)0.5 * (Real)n * nbar * crmax[c] * cdt + rem[c];
        const Real nsel_d = std::floor(ncand);
        rem[c] = ncand - nsel_d;
        uint64_t nsel = (uint64_t)nsel_d;
        if (nsel > 0xFFFFFFu) {
            status |= ST_CELL_OVERFLOW;
            nsel = 0xFFFFFFu;
        }
        counters[C_CANDIDATES] += nsel;
        for (uint32_t k = 0; k < nsel; ++k) {
            U4 r = draw(p.seed, gc, s, TAG_NTC_PAIR, k, 0);
            const uint32_t i = uindex(r[0], n);
            uint32_t j = uindex(r[1], n - 1);
            if (j >= i) j += 1;
            const Real R = (Real)u01f(r[2]);
            const uint32_t a = base + i, b = base + j;
            const Real dx = vx[a] - vx[b], dy = vy[a] - vy[b], dz = vz[a] - vz[b];
            const Real cr = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (cr > crmax[c]) crmax[c] = cr;
            if (cr > R * crmax[c]) {
                Real nv[3];
                if (!unit_vector(gc, s, k, nv)) {
                    status |= ST_SCATTER_CAP;
                    continue;
                }
                const Real cx = (vx[a] + vx[b]) * (Real)0.5;
                const Real cy = (vy[a] + vy[b]) * (Real)0.5;
                const Real cz = (vz[a] + vz[b]) * (Real)0.5;
                const Real h = cr * (Real)0.5;
                vx[a] = cx + h * nv[0]; vy[a] = cy + h * nv[1]; vz[a] = cz + h * nv[2];
                vx[b] = cx - h * nv[0]; vy[b] = cy - h * nv[1]; vz[b] = cz - h * nv[2];
                counters[C_COLLISIONS] += 1;
            }
        }
    }

    // Per-cell sums of 1, v, vv, vvv (Sec. 2.1 and Fig. 1: cumulative averages of the
    // hydrodynamic moments rho, u, P, Q).
    void sample_cell(uint32_t c) {
        double m[kNumMoments] = {};
        for (uint32_t i = cell_start[c]; i < cell_start[c + 1]; ++i) {
            const double v[3] = {(double)vx[i], (double)vy[i], (double)vz[i]};
            m[0] += 1.0;
            for (int a = 0; a < 3; ++a) m[1 + a] += v[a];
            int o = 4;
            for (int a = 0; a < 3; ++a)
                for (int b = a; b < 3; ++b) m[o++] += v[a] * v[b];
            for (int a = 0; a < 3; ++a)
                for (int b = a; b < 3; ++b)
                    for (int e = b; e < 3; ++e) m[o++] += v[a] * v[b] * v[e];
        }
        for (int k = 0; k < kNumMoments; ++k) acc[(size_t)c * kNumMoments + k] += m[k];
    }

    // The three phases of one step; step_once runs them in order.
    // The move of every particle; a streamwise slab's particles whose new cell is a
    // neighbour's go to the outbox.
    void phase_move() {
        const uint32_t s = (uint32_t)step;
        outbox[0].clear();
        outbox[1].clear();
        key_.assign(ntot(), kDeadKey);
        tag_.assign(ntot(), 0);
        for (int64_t c = 0; c < d.ncells; ++c) {
            const uint32_t gc = channel_cell(p, c);
            for (uint32_t i = cell_start[c]; i < cell_start[c + 1]; ++i) {
                const uint32_t rank = i - cell_start[c];
                const uint32_t gk = move_one(i, s, gc, rank);
                if (gk == kDeadKey) continue;
                tag_[i] = order_tag(gc, gk, rank);
                int dir;
                const int64_t lc = local_cell(gk, dir);
                if (lc >= 0) {
                    key_[i] = (uint32_t)lc;
                    continue;
                }
                Moved& o = outbox[dir];
                o.x.push_back(x[i]); o.y.push_back(y[i]); o.z.push_back(three_d() ? z[i] : (Real)0);
                o.vx.push_back(vx[i]); o.vy.push_back(vy[i]); o.vz.push_back(vz[i]);
                o.tag.push_back(tag_[i]);
                o.gkey.push_back(gk);
            }
        }
    }
    // The particles received from the neighbours join, and all are ordered by cell.
    void phase_accept_sort(const Moved* in, int nin) {
        for (int b = 0; b < nin; ++b)
            for (size_t k = 0; k < in[b].size(); ++k) {
                int dir;
                const int64_t lc = local_cell(in[b].gkey[k], dir);
                if (lc < 0) {
                    status |= ST_BAD_INPUT;
                    continue;
                }
                x.push_back(in[b].x[k]); y.push_back(in[b].y[k]);
                if (three_d()) z.push_back(in[b].z[k]);
                vx.push_back(in[b].vx[k]); vy.push_back(in[b].vy[k]); vz.push_back(in[b].vz[k]);
                key_.push_back((uint32_t)lc);
                tag_.push_back(in[b].tag[k]);
            }
        sort_by_cell(key_, tag_);
    }
    void phase_move_sort() {
        phase_move();
        phase_accept_sort(nullptr, 0);
    }
    void phase_collide() {
        const uint32_t s = (uint32_t)step;
        for (int64_t c = 0; c < d.ncells; ++c) collide_cell((uint32_t)c, s);
    }
    void phase_sample_advance() {
        const uint32_t s = (uint32_t)step;
        if (s % (uint32_t)p.sample_every == 0) {
            for (int64_t c = 0; c < d.ncells; ++c) sample_cell((uint32_t)c);
            nsamples += 1;
        }
        step += 1;
    }
    void step_once() {
        phase_move_sort();
        phase_collide();
        phase_sample_advance();
    }
};

}  // namespace ora
