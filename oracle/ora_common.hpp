// Oracle: common definitions (parameters, derived constants, Philox, lattices).
//
// TEST INFRASTRUCTURE ONLY. This directory is a plain, slow, CPU-only restatement of the
// DSMC-LBM mapping method of Di Staso, Clercx, Succi and Toschi (arXiv 1512.08042). It exists
// to check the CUDA library against the paper. Only the test suite, the smoke check and the
// CPU-baseline leg of the benchmark may load it; the product path never does. It shares no
// code, header, table or constant generator with the CUDA library.
//
// Units (the reading of the paper's Appendix A used throughout):
//   length   : DSMC cell size (cubic cells, App. A "length scale" L0 = dx_DSMC)
//   velocity : thermal speed c_th = sqrt(kT/m); the Hermite weight function then has unit
//              variance (Sec. 2.2, Eq. globalMax with T = 1)
//   time     : one DSMC step equals one LB step, T0 = (c_s/a) dx_LB with a = c_th
//              (App. A "time scale", isothermal reading of a)
//   density  : LB density 1 corresponds to `ppc` particles per DSMC cell
//              (App. A "mass scale", mass conserved at the coupling sites)
#pragma once
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace ora {

// ---------------------------------------------------------------------------------------
// Parameters. Field order is a binary interface with oracle.py (ctypes).
struct Params {
    uint32_t abi_version;
    int32_t ncx;           // DSMC cells across the channel, walls at x = 0 and x = ncx
    int32_t ncy;           // DSMC cells streamwise, periodic
    int32_t lb_ratio;      // LB nodes per DSMC cell per axis
    int32_t ppc;           // particles per cell at initialisation
    int32_t lattice;       // 39 (D3Q39, Hermite order 3) or 19 (D3Q19, order 2)
    int32_t real_bytes;    // 4 (float state) or 8 (double state)
    int32_t sample_every;  // moment sampling cadence in DSMC steps
    uint64_t seed;
    double kn;             // Knudsen number based on channel height
    double ma;             // Mach number of the no-slip centreline velocity, u_max / c_s
    double crmax_init;     // initial (sigma_T c_r)_max / sigma_T, in c_th units
    double capacity_factor;
    double T_K;            // temperature [K], SI reporting only
    double mass_kg;        // molecular mass [kg], SI reporting only
    int32_t lb_collision;  // 0 regularised BGK (Sec. 2), 1 plain BGK (Sec. 4)
    int32_t d2l_mode;      // 0 Grad to the lattice order (Sec. 2.1), 1 equilibrium (Eq. feq_dsmc)
    int32_t kn_profile;    // 1: Kn varies along the channel (kn_at)
    int32_t pad0;
    double kn_end;         // Kn at y = ncy / 2 when kn_profile = 1
    int32_t ncz;           // DSMC cells along z (periodic); 0 or 1: the quasi-2D slab
    int32_t accum_mode;    // moment sums: 0 FP64
    int32_t ncy_global;    // > 0: a streamwise slab of a channel of ncy_global rows
    int32_t y0;            // its first row in the channel
};

// Derived constants. Field order is a binary interface with oracle.py.
struct Derived {
    double r_lat;     // lattice scale: xi_a = r_lat * e_a in Hermite units (c/c_s)
    double cs_lat;    // lattice sound speed in lattice units, 1 / r_lat
    double H_lat;     // LB nodes across the channel
    double tau;       // BGK relaxation time, Eq. tau
    double dt;        // DSMC (= LB) time step in cell / c_th units
    double lambda;    // hard-sphere mean free path in DSMC cells, lambda = Kn * H
    double coll_dt;   // F_N sigma_T dt / V_c in the NTC count, Eq. collisionnumber
    double g_step;    // body-force velocity increment per step (Hermite units)
    double c_th_ms;   // sqrt(k T / m) in m/s
    int64_t ncells, nx, ny, nnodes, capacity;
    int32_t q, order;
    int32_t bin;   // particle slots per cell in the library's binned layout
    int32_t pad;
    int64_t nz;    // LB layers along z: 1 for the slab, ncz * lb_ratio in 3D
    int64_t ncz;   // DSMC cells along z: 1 for the slab
    int64_t yh;    // LB ghost rows below and above a streamwise slab's rows (0 otherwise)
    int64_t xcap;  // particles per exchange buffer of the library's slab layout
};

constexpr double kPi = 3.14159265358979323846;
constexpr double kBoltzmann = 1.380649e-23;

// Eq. tau for the lattice relaxation time; Eq. MFP read in DSMC cell units; the NTC factor
// of Eq. collisionnumber with F_N sigma_T / V_c = 1 / (sqrt(2) lambda ppc) because the
// number density is ppc F_N / V_c. The force is fixed by the no-slip parabola
// u_max = g H^2 / (8 nu) at u_max = Ma c_s (Sec. 3.1), nu = (tau - 1/2) c_s^2.
inline Derived derive(const Params& p) {
    Derived d{};
    d.r_lat = (p.lattice == 39) ? std::sqrt(1.5) : std::sqrt(3.0);
    d.cs_lat = 1.0 / d.r_lat;
    d.H_lat = (double)p.ncx * (double)p.lb_ratio;
    d.tau = std::sqrt(kPi / 8.0) * d.r_lat * p.kn * d.H_lat + 0.5;
    d.dt = d.cs_lat / (double)p.lb_ratio;
    d.lambda = p.kn * (double)p.ncx;
    d.coll_dt = d.dt / (std::sqrt(2.0) * d.lambda * (double)p.ppc);
    d.g_step = 8.0 * (d.tau - 0.5) * p.ma * d.cs_lat * d.cs_lat / (d.H_lat * d.H_lat);
    d.c_th_ms = std::sqrt(kBoltzmann * p.T_K / p.mass_kg);
    // 3D when ncz >= 2: cells (iz ncy + iy) ncx + ix, nodes (z ny + y) nx + x, periodic in z;
    // otherwise the quasi-2D slab of one cell and one LB layer
    d.ncz = p.ncz >= 2 ? p.ncz : 1;
    d.ncells = (int64_t)p.ncx * p.ncy * d.ncz;
    d.nx = (int64_t)p.ncx * p.lb_ratio;
    // a streamwise slab's lattice carries yh ghost rows below and above its own rows
    d.yh = p.ncy_global > 0 ? (p.lattice == 39 ? 3 : 1) : 0;
    d.ny = (int64_t)p.ncy * p.lb_ratio + 2 * d.yh;
    d.nz = p.ncz >= 2 ? d.ncz * p.lb_ratio : 1;
    d.nnodes = d.nx * d.ny * d.nz;
    d.bin = ((int32_t)std::ceil(p.capacity_factor * (double)p.ppc) + 31) / 32 * 32;
    d.capacity = d.ncells * (int64_t)d.bin;
    d.xcap = p.ncy_global > 0 ? (int64_t)p.ncx * d.ncz * d.bin : 0;
    d.q = p.lattice;
    d.order = (p.lattice == 39) ? 3 : 2;
    return d;
}

// Kn along the channel when kn_profile = 1: log-linear in the streamwise coordinate y (DSMC
// cell units, period ncy) from kn at y = 0 to kn_end at y = ncy / 2 and back,
// Kn(y) = kn (kn_end / kn)^s with s = 1 - |2 y / ncy - 1|. A DSMC cell takes the NTC factor
// of Eq. collisionnumber at its centre's Kn, an LB node the tau of Eq. tau at its own.
inline double kn_at(const Params& p, double y) {
    const double period = p.ncy_global > 0 ? (double)p.ncy_global : (double)p.ncy;
    const double s = 1.0 - std::fabs(2.0 * y / period - 1.0);
    return p.kn * std::exp(s * std::log(p.kn_end / p.kn));
}

// With the Kn profile: the NTC factor of Eq. collisionnumber (F_N sigma_T dt / V_c) of a DSMC
// cell in the channel's row iy, at the Kn of the cell's centre, and tau of Eq. tau of an LB
// node in the channel's LB row j, at the Kn of the row's centre.
inline double kn_cell_coll(const Params& p, const Derived& d, int64_t iy) {
    const double kn = kn_at(p, (double)iy + 0.5);
    return d.dt / (std::sqrt(2.0) * (kn * (double)p.ncx) * (double)p.ppc);
}
inline double kn_node_tau(const Params& p, const Derived& d, int64_t j) {
    const double kn = kn_at(p, ((double)j + 0.5) / (double)p.lb_ratio);
    return std::sqrt(kPi / 8.0) * d.r_lat * kn * d.H_lat + 0.5;
}

// A streamwise slab (ncy_global > 0) holds the channel's rows [y0, y0 + ncy): the channel's
// row of the slab's row iy, the channel's cell id of the slab's cell c = (iz ncy + iy) ncx + ix,
// and the channel's LB row of the slab's lattice row j (its yh ghost rows hold the
// neighbours' rows, periodically). For a context that holds the whole channel these are
// identities.
inline int64_t channel_rows(const Params& p) { return p.ncy_global > 0 ? p.ncy_global : p.ncy; }
inline uint32_t channel_cell(const Params& p, int64_t c) {
    const int64_t plane = (int64_t)p.ncx * p.ncy;
    const int64_t iz = c / plane, r = c % plane;
    const int64_t y0 = p.ncy_global > 0 ? p.y0 : 0;
    return (uint32_t)((iz * channel_rows(p) + y0 + r / p.ncx) * p.ncx + r % p.ncx);
}
inline int64_t channel_lb_row(const Params& p, const Derived& d, int64_t j) {
    const int64_t rows = channel_rows(p) * p.lb_ratio;
    const int64_t y0 = p.ncy_global > 0 ? p.y0 : 0;
    return (((y0 * p.lb_ratio + j - d.yh) % rows) + rows) % rows;
}

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 32x32->64 multiplies; the key is bumped by the Weyl constants
// between rounds.
using U4 = std::array<uint32_t, 4>;

inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = M0 * (uint64_t)c[0];
        uint64_t p1 = M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = U4{hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0};
    }
    return c;
}

// Purpose tags of the counter layout (entity, step, tag << 24 | sub-index, block).
enum Tag : uint32_t {
    TAG_INIT_POS = 1,
    TAG_INIT_VEL = 2,
    TAG_WALL = 3,
    TAG_NTC_PAIR = 4,
    TAG_NTC_SCAT = 5,
    TAG_L2D_VEL = 6,
    TAG_L2D_POS = 7,
    TAG_L2D_ROUND = 8,
};

inline U4 draw(uint64_t seed, uint32_t entity, uint32_t step, uint32_t tag, uint32_t sub,
               uint32_t block) {
    return philox4x32_10(U4{entity, step, (tag << 24) | (sub & 0xFFFFFFu), block},
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform on [0,1) with 24 bits, exact in float.
inline float u01f(uint32_t r) { return (float)(r >> 8) * 0x1p-24f; }
// Uniform on (0,1), for logarithms.
inline double u01open(uint32_t r) { return ((double)r + 0.5) * 0x1p-32; }
// Uniform on [0,1) with 32 bits.
inline double u01d(uint32_t r) { return (double)r * 0x1p-32; }
// Integer uniform on [0, n) by the 64-bit multiply-shift map.
inline uint32_t uindex(uint32_t r, uint32_t n) { return (uint32_t)(((uint64_t)r * n) >> 32); }

// Box-Muller transform (Box and Muller 1958), the sampler Table 1 step 4 names.
inline void box_muller(uint32_t r1, uint32_t r2, double& n1, double& n2) {
    double rad = std::sqrt(-2.0 * std::log(u01open(r1)));
    double th = 6.283185307179586 * u01open(r2);
    n1 = rad * std::cos(th);
    n2 = rad * std::sin(th);
}

// Float elementary functions used by the float state path. They are written out from their
// series so that every IEEE operation is fixed and the same float results follow on any
// machine that rounds each operation (no contraction):
//   ln x: x = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s), s = (m-1)/(m+1),
//         atanh s = s + s^3/3 + ... + s^11/11 (Abramowitz & Stegun 4.6.22), ln 2 split into
//         a float-exact head and a small tail;
//   sin, cos of 2 pi u (u in [0,1) with 24 bits): exact quadrant and octant reduction on u,
//         then Taylor series of sin and cos on [0, pi/4] (A&S 4.3.65, 4.3.66).
inline float ln_f(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    const uint32_t mb = (b & 0x7FFFFFu) | 0x3F800000u;
    float m;
    std::memcpy(&m, &mb, 4);
    if (m > 1.41421356f) {
        m = m * 0.5f;
        e += 1;
    }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float t = 1.0f / 11.0f;
    t = t * s2 + 1.0f / 9.0f;
    t = t * s2 + 1.0f / 7.0f;
    t = t * s2 + 1.0f / 5.0f;
    t = t * s2 + 1.0f / 3.0f;
    t = t * s2 + 1.0f;
    const float lnm = 2.0f * s * t;
    const float fe = (float)e;
    return fe * 0.693145751953125f + (fe * 1.4286068203e-06f + lnm);
}

inline void sincos2pi_f(float u, float& sn, float& cs) {
    const float t = 4.0f * u;
    const float k = std::floor(t);
    const float f = t - k;
    const int q = (int)k & 3;
    const bool swap = f > 0.5f;
    const float g = swap ? 1.0f - f : f;
    const float phi = g * 1.57079637f;
    const float p2 = phi * phi;
    float ps = 1.0f / 362880.0f;
    ps = ps * p2 - 1.0f / 5040.0f;
    ps = ps * p2 + 1.0f / 120.0f;
    ps = ps * p2 - 1.0f / 6.0f;
    ps = ps * p2 + 1.0f;
    const float sp = phi * ps;
    float pc = -1.0f / 3628800.0f;
    pc = pc * p2 + 1.0f / 40320.0f;
    pc = pc * p2 - 1.0f / 720.0f;
    pc = pc * p2 + 1.0f / 24.0f;
    pc = pc * p2 - 0.5f;
    pc = pc * p2 + 1.0f;
    const float sa = swap ? pc : sp;
    const float ca = swap ? sp : pc;
    switch (q) {
        case 0: sn = sa; cs = ca; break;
        case 1: sn = ca; cs = -sa; break;
        case 2: sn = -sa; cs = -ca; break;
        default: sn = -ca; cs = sa; break;
    }
}

// A pair of unit normals (Box-Muller) and the speed of a particle re-emitted by a diffuse
// wall (sqrt(-2 ln U), the flux-weighted Maxwellian), in the state precision. Float: 24-bit
// uniforms, U1 in (0, 1]; double: libm in double with 32-bit uniforms.
template <class Real>
inline void gauss_pair(uint32_t r1, uint32_t r2, Real& n1, Real& n2);
template <>
inline void gauss_pair<float>(uint32_t r1, uint32_t r2, float& n1, float& n2) {
    const float u1 = (float)((r1 >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(r2 >> 8) * 0x1p-24f;
    const float rad = std::sqrt(-2.0f * ln_f(u1));
    float sn, cs;
    sincos2pi_f(u2, sn, cs);
    n1 = rad * cs;
    n2 = rad * sn;
}
template <>
inline void gauss_pair<double>(uint32_t r1, uint32_t r2, double& n1, double& n2) {
    box_muller(r1, r2, n1, n2);
}
template <class Real>
inline Real wall_speed(uint32_t r);
template <>
inline float wall_speed<float>(uint32_t r) {
    const float u = (float)((r >> 8) + 1u) * 0x1p-24f;
    return std::sqrt(-2.0f * ln_f(u));
}
template <>
inline double wall_speed<double>(uint32_t r) {
    return std::sqrt(-2.0 * std::log(u01open(r)));
}

// ---------------------------------------------------------------------------------------
// Lattices. The paper names D3Q19 and the 39-speed sixth-order-isotropic Gauss-Hermite set
// (Sec. 1, Sec. 3.1) without listing them; these are the Shan-Yuan-Chen (2006) sets, pinned
// by the quadrature-degree tests. Row order is the population layout of the library.
struct Lattice {
    int q;
    double r;
    std::vector<std::array<int, 3>> e;
    std::vector<double> w;
    std::vector<std::array<double, 3>> xi;  // r * e, Hermite units
};

inline Lattice make_lattice(int q) {
    Lattice L;
    L.q = q;
    auto add = [&](int x, int y, int z, double w) {
        L.e.push_back({x, y, z});
        L.w.push_back(w);
    };
    if (q == 39) {
        L.r = std::sqrt(1.5);
        add(0, 0, 0, 1.0 / 12.0);
        const int s1[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        for (auto& v : s1) add(v[0], v[1], v[2], 1.0 / 12.0);
        const int s3[8][3] = {{1, 1, 1},  {-1, 1, 1},  {1, -1, 1},  {-1, -1, 1},
                              {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
        for (auto& v : s3) add(v[0], v[1], v[2], 1.0 / 27.0);
        for (auto& v : s1) add(2 * v[0], 2 * v[1], 2 * v[2], 2.0 / 135.0);
        const int s8[12][3] = {{2, 2, 0},  {-2, 2, 0},  {2, -2, 0},  {-2, -2, 0},
                               {2, 0, 2},  {-2, 0, 2},  {2, 0, -2},  {-2, 0, -2},
                               {0, 2, 2},  {0, -2, 2},  {0, 2, -2},  {0, -2, -2}};
        for (auto& v : s8) add(v[0], v[1], v[2], 1.0 / 432.0);
        for (auto& v : s1) add(3 * v[0], 3 * v[1], 3 * v[2], 1.0 / 1620.0);
    } else {
        L.r = std::sqrt(3.0);
        add(0, 0, 0, 1.0 / 3.0);
        const int s1[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        for (auto& v : s1) add(v[0], v[1], v[2], 1.0 / 18.0);
        const int s2[12][3] = {{1, 1, 0},  {-1, 1, 0},  {1, -1, 0},  {-1, -1, 0},
                               {1, 0, 1},  {-1, 0, 1},  {1, 0, -1},  {-1, 0, -1},
                               {0, 1, 1},  {0, -1, 1},  {0, 1, -1},  {0, -1, -1}};
        for (auto& v : s2) add(v[0], v[1], v[2], 1.0 / 36.0);
    }
    for (auto& e : L.e) L.xi.push_back({L.r * e[0], L.r * e[1], L.r * e[2]});
    return L;
}

// ---------------------------------------------------------------------------------------
// Hermite polynomials (Grad 1949; Shan, Yuan, Chen 2006), Sec. 2 Eq. series:
// H0 = 1, H1_i = xi_i, H2_ij = xi_i xi_j - d_ij, H3_ijk = xi_i xi_j xi_k - xi_i d_jk
// - xi_j d_ik - xi_k d_ij.
inline double kd(int i, int j) { return i == j ? 1.0 : 0.0; }
inline double H2(const double* x, int i, int j) { return x[i] * x[j] - kd(i, j); }
inline double H3(const double* x, int i, int j, int k) {
    return x[i] * x[j] * x[k] - x[i] * kd(j, k) - x[j] * kd(i, k) - x[k] * kd(i, j);
}

// Full tensors, no symmetry packing.
struct Coeffs {
    double a0;
    double a1[3];
    double a2[3][3];
    double a3[3][3][3];
};

// Truncated series of Eq. seriestrunc divided by the weight: sum_{n<=N} a^(n) H^(n)(xi) / n!
inline double hermite_series(const Coeffs& a, const double* x, int order) {
    double s = a.a0;
    for (int i = 0; i < 3; ++i) s += a.a1[i] * x[i];
    double s2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s2 += a.a2[i][j] * H2(x, i, j);
    s += 0.5 * s2;
    if (order >= 3) {
        double s3 = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) s3 += a.a3[i][j][k] * H3(x, i, j, k);
        s += s3 / 6.0;
    }
    return s;
}

// Eq. coefficients_LBM: a^(n) = sum_a f_a H^(n)(xi_a).
inline Coeffs project(const Lattice& L, const double* f) {
    Coeffs a{};
    for (int q = 0; q < L.q; ++q) {
        const double* x = L.xi[q].data();
        a.a0 += f[q];
        for (int i = 0; i < 3; ++i) {
            a.a1[i] += f[q] * x[i];
            for (int j = 0; j < 3; ++j) {
                a.a2[i][j] += f[q] * H2(x, i, j);
                for (int k = 0; k < 3; ++k) a.a3[i][j][k] += f[q] * H3(x, i, j, k);
            }
        }
    }
    return a;
}

// Status bits of the sticky status word (same meanings as the library's).
enum StatusBit : uint32_t {
    ST_CAPACITY = 1u << 0,
    ST_BOUNCE_CAP = 1u << 1,
    ST_SCATTER_CAP = 1u << 2,
    ST_SAMPLING_CAP = 1u << 3,
    ST_CELL_OVERFLOW = 1u << 4,
    ST_BAD_INPUT = 1u << 5,
};

}  // namespace ora
