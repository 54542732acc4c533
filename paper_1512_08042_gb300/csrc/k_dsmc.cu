// DSMC kernels: initialisation, move with diffuse isothermal walls and binning by cell,
// and the per-cell stable ordering, no-time-counter hard-sphere collisions and
// Hermite-moment sampling.
//
// Particles live in per-cell bins of `bin` slots (cell c owns slots [c bin, (c+1) bin) of
// each state array, count[c] in use) and ping-pong between two halves. One DSMC step (the
// NTC order of Bird that the paper uses in Sec. 5: move, index, collide, sample) is two
// launches:
//   k_move     one warp per source cell: body-force kick, free flight, diffuse wall
//              re-emission (Sec. 3.1), periodic wrap, new cell; the moved particle is written
//              as one record (x, y, vx, vy, vz) at its origin slot of the `moved` scratch, and
//              the slot is appended to the tag list of its new cell's bin by a warp-aggregated
//              atomic.
//   k_collide  32 consecutive cells per block, a group of 8 lanes per cell: the cell's tags
//              are put in stable order (ascending origin slot = origin cell, then rank in it:
//              a bitonic sort in registers), the records are gathered into the bin of the
//              other half (positions) and a shared-memory pool (velocities), the NTC
//              candidates of all 32 cells are drawn by the whole block and applied by one
//              warp with a lane per cell (Eq. collisionnumber), and the sums 1, v, vv, vvv are
//              added to the FP64 cumulative sums of the cell (Sec. 2.1, Fig. 1). The last
//              block to finish advances the step counters.
// This file is compiled without FMA contraction so that positions, cell keys, pair choices
// and post-collision velocities are the IEEE float (or double) results of the written
// expressions.
#include <cstring>

#include "hyb_internal.cuh"

namespace hyb {

namespace {

template <typename Real>
__device__ __forceinline__ void reemit(uint64_t seed, uint32_t cell, uint32_t rank, uint32_t s,
                                       int bounce, Real sign, Real& ux, Real& uy, Real& uz) {
    const uint4 r = draw(seed, cell, s, TAG_WALL, (rank << 3) | (uint32_t)bounce, 0);
    const Real vn = wall_speed<Real>(r.x);
    Real t1, t2;
    gauss_pair<Real>(r.y, r.z, t1, t2);
    ux = sign * vn;
    uy = t1;
    uz = t2;
}

// Isotropic unit vector (Marsaglia 1972) from the NTC scattering stream of candidate k.
template <typename Real>
__device__ __forceinline__ int unit_vector(uint64_t seed, uint32_t c, uint32_t s, uint32_t k, Real& nx,
                                           Real& ny, Real& nz) {
    for (int blk = 0; blk < kMaxScatterBlocks; ++blk) {
        const uint4 r = draw(seed, c, s, TAG_NTC_SCAT, k, (uint32_t)blk);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const Real u1 = (Real)2 * (Real)u01f(w[2 * h]) - (Real)1;
            const Real u2 = (Real)2 * (Real)u01f(w[2 * h + 1]) - (Real)1;
            const Real ss = u1 * u1 + u2 * u2;
            if (ss < (Real)1) {
                const Real a = (Real)2 * sqrt((Real)1 - ss);
                nx = u1 * a;
                ny = u2 * a;
                nz = (Real)1 - (Real)2 * ss;
                return 1;
            }
        }
    }
    nx = ny = nz = (Real)0;
    return 0;
}

// ---------------------------------------------------------------------------------------
template <typename Real>
__global__ void k_init_particles(DsmcArgs<Real> a) {
    const int64_t n = (int64_t)a.ncells * a.ppc;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(s / a.ppc), k = (uint32_t)(s % a.ppc);
        const int ix = (int)(c % (uint32_t)a.ncx), iy = (int)((c / (uint32_t)a.ncx) % (uint32_t)a.ncy);
        const int64_t slot = (int64_t)c * a.bin + k;
        const uint4 rp = draw(a.seed, c, 0, TAG_INIT_POS, k, 0);
        a.dx[slot] = (Real)ix + (Real)u01f(rp.x);
        a.dy[slot] = (Real)iy + (Real)u01f(rp.y);
        if (a.ncz) a.dz[slot] = (Real)(c / ((uint32_t)a.ncx * (uint32_t)a.ncy)) + (Real)u01f(rp.z);
        const uint4 rv = draw(a.seed, c, 0, TAG_INIT_VEL, k, 0);
        Real n0, n1, n2, n3;
        gauss_pair<Real>(rv.x, rv.y, n0, n1);
        gauss_pair<Real>(rv.z, rv.w, n2, n3);
        a.dvx[slot] = n0;
        a.dvy[slot] = n1;
        a.dvz[slot] = n2;
    }
}

template <typename Real>
__global__ void k_init_cells(DsmcArgs<Real> a) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        a.count_d[c] = (uint32_t)a.ppc;
        a.count_s[c] = 0;
        a.crmax[c] = (Real)a.crmax_init;
        a.rem[c] = (Real)0;
        a.nbar_sum[c] = 0u;
        for (int m = 0; m < kMoments; ++m) a.acc[c * kMoments + m] = 0.0;
        if (c == 0) {
            for (int w = 0; w < CTRL_WORDS; ++w) a.ctrl[w] = 0;
            a.ctrl[CTRL_NTOT] = (uint32_t)((int64_t)a.ncells * a.ppc);
            for (int w = 0; w < HYB_NCOUNTERS; ++w) a.counters[w] = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Moved-particle records: 8 Real per origin slot (x, y, vx, vy, vz, 3 unused), written whole
// by the move and read by the collide with one 32-byte sector per particle (FP32).
__device__ __forceinline__ void rec_store(float* rec, int64_t i, float x, float y, float u, float v,
                                          float w, float z = 0.0f) {
    float4* p = reinterpret_cast<float4*>(rec) + 2 * i;
    p[0] = make_float4(x, y, u, v);
    p[1] = make_float4(w, z, 0.0f, 0.0f);
}
__device__ __forceinline__ void rec_store(double* rec, int64_t i, double x, double y, double u,
                                          double v, double w, double z = 0.0) {
    double2* p = reinterpret_cast<double2*>(rec) + 4 * i;
    p[0] = make_double2(x, y);
    p[1] = make_double2(u, v);
    p[2] = make_double2(w, z);
}
// Z3: also the z position (3D), stored beside vz.
template <bool Z3>
__device__ __forceinline__ void rec_load(const float* rec, int64_t i, float& x, float& y, float& u,
                                         float& v, float& w, float& z) {
    const float4* p = reinterpret_cast<const float4*>(rec) + 2 * i;
    const float4 a = p[0];
    x = a.x;
    y = a.y;
    u = a.z;
    v = a.w;
    if constexpr (Z3) {
        const float2 b = reinterpret_cast<const float2*>(p + 1)[0];
        w = b.x;
        z = b.y;
    } else {
        w = reinterpret_cast<const float*>(p + 1)[0];
    }
}
template <bool Z3>
__device__ __forceinline__ void rec_load(const double* rec, int64_t i, double& x, double& y,
                                         double& u, double& v, double& w, double& z) {
    const double2* p = reinterpret_cast<const double2*>(rec) + 4 * i;
    const double2 a = p[0], b = p[1];
    x = a.x;
    y = a.y;
    u = b.x;
    v = b.y;
    if constexpr (Z3) {
        const double2 c = p[2];
        w = c.x;
        z = c.y;
    } else {
        w = reinterpret_cast<const double*>(p + 2)[0];
    }
}

// ---------------------------------------------------------------------------------------
// Move (kick, drift, walls, wrap) and binning into the other half.

// Flight of a particle whose straight flight crosses a wall: it is re-emitted from the wall
// (diffuse, isothermal), possibly more than once, for the rest of the step.
template <typename Real, bool Z3 = false>
__device__ __forceinline__ void wall_flight(uint64_t seed, uint32_t c, uint32_t k, uint32_t s, Real H,
                                            Real dt, Real& px, Real& py, Real& ux, Real& uy,
                                            Real& uz, uint32_t& hits, uint32_t& caps, Real& pz) {
    Real t = dt;
    for (int b = 0;; ++b) {
        const Real xn = px + ux * t;
        const bool left = xn < (Real)0;
        const bool right = xn > H;
        if (!left && !right) {
            px = xn;
            py = py + uy * t;
            if constexpr (Z3) pz = pz + uz * t;
            break;
        }
        if (b == kMaxBounces) {
            caps += 1;
            px = left ? (Real)0 : H;
            py = py + uy * t;
            if constexpr (Z3) pz = pz + uz * t;
            break;
        }
        hits += 1;
        const Real th = left ? px / (-ux) : (H - px) / ux;
        py = py + uy * th;
        if constexpr (Z3) pz = pz + uz * th;
        px = left ? (Real)0 : H;
        t = t - th;
        if (t < (Real)0) t = (Real)0;
        reemit(seed, c, k, s, b, left ? (Real)1 : (Real)-1, ux, uy, uz);
    }
}

// Exact widening of a float to double on the integer pipe (the FP64 pipe is slow on this
// part): a normal float's sign, exponent rebiased from 127 to 1023 and mantissa shifted to
// the top of the 52-bit field (IEEE 754 binary32 and binary64 formats). Zeros, subnormals,
// infinities and NaNs take the plain conversion.
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                          ((uint64_t)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double d) { return d; }

// Periodic wrap of v into [0, period).
template <typename Real>
__device__ __forceinline__ Real wrap_periodic(Real v, Real period) {
    if (v < (Real)0 || v >= period) {
        v = v - period * floor(v / period);
        if (v < (Real)0) v = v + period;
        if (v >= period) v = v - period;
    }
    return v;
}

// Periodic wrap of y (and z in 3D) and the cell key (iz ncy + iy) ncx + ix of a moved particle.
template <typename Real, bool Z3 = false>
__device__ __forceinline__ uint32_t cell_key(const DsmcArgs<Real>& a, Real L, Real px, Real& py,
                                             Real& pz) {
    py = wrap_periodic(py, L);
    int ix = (int)floor(px), iy = (int)floor(py);
    ix = ix < 0 ? 0 : (ix > a.ncx - 1 ? a.ncx - 1 : ix);
    iy = iy < 0 ? 0 : (iy > a.ncy - 1 ? a.ncy - 1 : iy);
    int iz = 0;
    if constexpr (Z3) {
        pz = wrap_periodic(pz, (Real)a.ncz);
        iz = (int)floor(pz);
        iz = iz < 0 ? 0 : (iz > a.ncz - 1 ? a.ncz - 1 : iz);
    }
    return (uint32_t)((iz * a.ncy + iy) * a.ncx + ix);
}

// Appends the active lanes' two slots to the bins of their new cells: lanes bound for the
// same cell share one atomic, and each gets arrival = base + rank among them. The atomics
// of both slots are in flight before either result is used.
__device__ __forceinline__ void bin_arrival2(uint32_t* __restrict__ count, uint32_t key1, bool act1,
                                             uint32_t key2, bool act2, unsigned lane, uint32_t& arr1,
                                             uint32_t& arr2) {
    // inactive lanes match among themselves under a key no cell has
    const unsigned peers1 = __match_any_sync(kFull, act1 ? key1 : 0xFFFFFFFFu);
    const unsigned peers2 = __match_any_sync(kFull, act2 ? key2 : 0xFFFFFFFFu);
    const int lead1 = __ffs(peers1) - 1, lead2 = __ffs(peers2) - 1;
    uint32_t b1 = 0, b2 = 0;
    if (act1 && (int)lane == lead1) b1 = atomicAdd(&count[key1], (uint32_t)__popc(peers1));
    if (act2 && (int)lane == lead2) b2 = atomicAdd(&count[key2], (uint32_t)__popc(peers2));
    b1 = __shfl_sync(kFull, b1, lead1);
    b2 = __shfl_sync(kFull, b2, lead2);
    const unsigned below = (1u << lane) - 1u;
    arr1 = b1 + (uint32_t)__popc(peers1 & below);
    arr2 = b2 + (uint32_t)__popc(peers2 & below);
}

// One source cell, by one warp; the first 64 particles of the cell are handled two per
// lane, loads, flights and binning atomics of both in flight together.
template <typename Real, bool Z3>
__device__ __forceinline__ void move_cell(const DsmcArgs<Real>& a, int c, unsigned lane) {
    const uint32_t s = a.ctrl[CTRL_STEP];
    if (c == 0 && lane == 0) a.ctrl[CTRL_NTOT] = 0;  // the collide recounts
    const Real H = (Real)a.ncx, L = (Real)a.ncy;
    const Real g = a.g_r, dt = a.dt_r;
    const uint32_t bin = (uint32_t)a.bin;
    // the arrays do not overlap: loads of the next slots need not wait for earlier stores
    const Real* __restrict__ sx = a.sx;
    const Real* __restrict__ sy = a.sy;
    const Real* __restrict__ svx = a.svx;
    const Real* __restrict__ svy = a.svy;
    const Real* __restrict__ svz = a.svz;
    Real* __restrict__ rec = a.rec;
    uint32_t* __restrict__ tag = a.tag;
    uint32_t* __restrict__ cnt = a.count_d;
    uint32_t hits = 0, caps = 0, lost = 0;
    {
        uint32_t n = a.count_s[c];
        if (n > bin) n = bin;
        const int64_t base = (int64_t)c * bin;
        for (uint32_t k0 = 0; k0 == 0 || k0 < n; k0 += 64) {
            const uint32_t k1 = k0 + lane, k2 = k1 + 32;
            const bool act1 = k1 < n, act2 = k2 < n;
            Real p1[5] = {0, 0, 0, 0, 0}, p2[5] = {0, 0, 0, 0, 0};
            Real z1 = 0, z2 = 0;  // 3D only
            // the loads need only the bin size, not the count, so they travel with it
            const bool in1 = k1 < bin, in2 = k2 < bin;
            if (in1) {
                p1[0] = sx[base + k1];
                p1[1] = sy[base + k1];
                p1[2] = svx[base + k1];
                p1[3] = svy[base + k1];
                p1[4] = svz[base + k1];
                if constexpr (Z3) z1 = a.sz[base + k1];
            }
            if (in2) {
                p2[0] = sx[base + k2];
                p2[1] = sy[base + k2];
                p2[2] = svx[base + k2];
                p2[3] = svy[base + k2];
                p2[4] = svz[base + k2];
                if constexpr (Z3) z2 = a.sz[base + k2];
            }
            // kick and straight flight; flights that cross a wall are redone below
            p1[3] = p1[3] + g;
            p2[3] = p2[3] + g;
            const Real xn1 = p1[0] + p1[2] * dt, xn2 = p2[0] + p2[2] * dt;
            const bool wall1 = act1 && !(xn1 >= (Real)0 && xn1 <= H);
            const bool wall2 = act2 && !(xn2 >= (Real)0 && xn2 <= H);
            if (!wall1) {
                p1[0] = xn1;
                p1[1] = p1[1] + p1[3] * dt;
                if constexpr (Z3) z1 = z1 + p1[4] * dt;
            }
            if (!wall2) {
                p2[0] = xn2;
                p2[1] = p2[1] + p2[3] * dt;
                if constexpr (Z3) z2 = z2 + p2[4] * dt;
            }
            if (__any_sync(kFull, wall1 || wall2)) {
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    if (h == 0 ? wall1 : wall2) {
                        Real q[5];
#pragma unroll
                        for (int i = 0; i < 5; ++i) q[i] = h == 0 ? p1[i] : p2[i];
                        Real qz = h == 0 ? z1 : z2;
                        wall_flight<Real, Z3>(a.seed, (uint32_t)c, h == 0 ? k1 : k2, s, H, dt, q[0],
                                              q[1], q[2], q[3], q[4], hits, caps, qz);
                        if (h == 0)
                            z1 = qz;
                        else
                            z2 = qz;
#pragma unroll
                        for (int i = 0; i < 5; ++i) {
                            if (h == 0)
                                p1[i] = q[i];
                            else
                                p2[i] = q[i];
                        }
                    }
                }
            }
            const uint32_t key1 = act1 ? cell_key<Real, Z3>(a, L, p1[0], p1[1], z1) : 0u;
            const uint32_t key2 = act2 ? cell_key<Real, Z3>(a, L, p2[0], p2[1], z2) : 0u;
            uint32_t arr1, arr2;
            bin_arrival2(cnt, key1, act1, key2, act2, lane, arr1, arr2);
            if (act1) {
                rec_store(rec, base + k1, p1[0], p1[1], p1[2], p1[3], p1[4], z1);
                if (arr1 < bin)
                    tag[(int64_t)key1 * bin + arr1] = (uint32_t)(base + k1);
                else
                    lost += 1;
            }
            if (act2) {
                rec_store(rec, base + k2, p2[0], p2[1], p2[2], p2[3], p2[4], z2);
                if (arr2 < bin)
                    tag[(int64_t)key2 * bin + arr2] = (uint32_t)(base + k2);
                else
                    lost += 1;
            }
        }
    }
    if (__any_sync(kFull, (hits | caps | lost) != 0u)) {  // cells at a wall, or overflow
        hits = __reduce_add_sync(kFull, hits);
        caps = __reduce_add_sync(kFull, caps);
        lost = __reduce_add_sync(kFull, lost);
        if (lane == 0) {
            if (hits) atomicAdd(&a.counters[HYB_C_WALL_HITS], (unsigned long long)hits);
            if (caps) {
                atomicAdd(&a.counters[HYB_C_BOUNCE_CAP], (unsigned long long)caps);
                atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BOUNCE_CAP);
            }
            if (lost) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_CAPACITY);
        }
    }
}

// One warp per source cell (the cells of all replicas in the batch form).
template <typename Real, bool BATCH, bool Z3 = false>
__global__ void __launch_bounds__(256, 4) k_move(Launch<DsmcArgs<Real>> L) {
    pdl_begin();
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gw; u < L.total; u += nw) {
        if constexpr (BATCH) {
            const int r = replica_of(L.pre, L.nrep, u);
            move_cell<Real, Z3>(L.tab[r], (int)(u - L.pre[r]), lane);
        } else {
            move_cell<Real, Z3>(L.one, (int)u, lane);
        }
    }
}

// ---------------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------------
// Collide: a group of G lanes per cell, 32 / G cells per warp. Every instruction of the
// serial NTC chain then advances 32 / G cells at once. All loops that contain shuffles have
// warp-uniform trip counts (groups whose cell has less work are masked), so every shuffle is
// executed by the full warp.
constexpr int kGroup = 8;

template <typename Real>
struct CollideCfg {
    static constexpr int MINB = sizeof(Real) == 4 ? 4 : 2;  // resident blocks per SM
};
constexpr int kCollideWarps = 8;  // 32 cells per block
constexpr int kChainSteps = 16;   // candidates per cell drawn per pass of the NTC phase

// Ascending bitonic sort of G R keys held by the G lanes of a group, R per lane, in blocked
// order: key r of group lane l is at position (r % B) + B l + B G (r / B). Exchanges between
// positions less than B apart, or at least B G apart, stay in the lane's registers; the
// others are shuffles between the lanes of the group. Constant trip counts: the keys stay
// in registers.
template <int G, int R, int B>
__device__ __forceinline__ void bitonic_blocked(uint32_t (&v)[R]) {
    static_assert(R % B == 0, "whole blocks of B keys per lane");
    constexpr int N = G * R;
    const int gl = (int)(lane_id() % G);
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < B || j >= B * G) {
                const int jr = j < B ? j : j / G;  // distance in registers
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int o = r ^ jr;
                    if (r < o) {
                        const int pos = (r % B) + B * gl + B * G * (r / B);
                        const bool asc = (pos & k) == 0;
                        const uint32_t lo = min(v[r], v[o]), hi = max(v[r], v[o]);
                        v[r] = asc ? lo : hi;
                        v[o] = asc ? hi : lo;
                    }
                }
            } else {
                const int jl = j / B;  // distance in lanes
                const bool lower = (gl & jl) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t o = __shfl_xor_sync(kFull, v[r], jl);
                    const int pos = (r % B) + B * gl + B * G * (r / B);
                    const bool asc = (pos & k) == 0;
                    v[r] = (lower == asc) ? min(v[r], o) : max(v[r], o);
                }
            }
        }
    }
}

// Writes the sorted keys of blocked positions below n to st and reads back into v the keys
// of positions gl + G r (the order in which the group gathers); every lane of the warp
// calls it.
template <int G, int R, int B>
__device__ __forceinline__ void blocked_to_strided(uint32_t (&v)[R], uint32_t* st, uint32_t n, int gl) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t pos = (uint32_t)((r % B) + B * gl + B * G * (r / B));
        if (pos < n) st[pos] = v[r];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t k = (uint32_t)(gl + G * r);
        v[r] = k < n ? st[k] : 0u;
    }
}

// Gathers the particles of sorted positions k = gl + G r (r < RR) from the records of the
// origin slots src[r]: positions into the cell's bin of the other half, velocities into
// shared memory. The record, position and shared-memory pointers are declared free of
// aliasing, so the loads of all slots can be in flight before the first store.
template <typename Real, int G, int RR, bool Z3>
__device__ __forceinline__ void gather_slots(const Real* __restrict__ rec, Real* __restrict__ dx,
                                             Real* __restrict__ dy, Real* __restrict__ dz, int gl,
                                             uint32_t n, const uint32_t* src, Real* __restrict__ vx,
                                             Real* __restrict__ vy, Real* __restrict__ vz) {
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        const uint32_t k = (uint32_t)(gl + G * r);
        if (k < n) {
            Real px, py, ux, uy, uz, pz;
            rec_load<Z3>(rec, (int64_t)src[r], px, py, ux, uy, uz, pz);
            dx[k] = px;
            dy[k] = py;
            if constexpr (Z3) dz[k] = pz;
            vx[k] = ux;
            vy[k] = uy;
            vz[k] = uz;
        }
    }
}

// The block of 32 consecutive cells `blk` (of nblk) of one context.
template <typename Real, bool Z3>
__device__ __forceinline__ void collide_block(const DsmcArgs<Real>& a, uint32_t pool, int blk,
                                              int nblk) {
    constexpr int G = kGroup;
    constexpr int CPW = 32 / G;           // cells per warp in phases A and C
    constexpr int WARPS = kCollideWarps;
    constexpr int NC = WARPS * CPW;       // cells per block (one chain lane each in phase B)
    constexpr int SMALL = 64;             // cells up to this size are sorted in registers
    constexpr int R = SMALL / G;
    constexpr int KC = kChainSteps;       // candidates per cell drawn per pass of phase B
    static_assert(NC == 32, "phase B runs one lane per cell of the block in one warp");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_n[NC], s_off[NC], s_nsel[NC];
    __shared__ Real s_cm[NC];
    __shared__ uint32_t s_fits;
    __shared__ unsigned long long s_cnt[WARPS][2];
    __shared__ uint32_t s_live[WARPS], s_flags[WARPS];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int grp = (int)lane / G, gl = (int)lane % G;
    const int gi = w * CPW + grp;  // the group's cell within the block
    const uint32_t bin = (uint32_t)a.bin;
    // shared memory: the block's pool of vx, vy, vz (Real) and tags (u32), `pool` slots each,
    // then the candidates of one pass of phase B
    Real* pv = reinterpret_cast<Real*>(smem_raw);
    uint32_t* pst = reinterpret_cast<uint32_t*>(pv + 3 * (size_t)pool);
    uint32_t* c_ij = pst + pool;
    Real* c_R = reinterpret_cast<Real*>(c_ij + NC * KC);
    Real* c_nx = c_R + NC * KC;
    Real* c_ny = c_nx + NC * KC;
    Real* c_nz = c_ny + NC * KC;
    const uint32_t s = a.ctrl[CTRL_STEP];
    const bool do_sample = (s % (uint32_t)a.sample_every) == 0u;
    const Real coll_dt = a.coll_r;
    unsigned long long ncand_tot = 0, ncoll_tot = 0;
    uint32_t flags = 0, nlive = 0;

    const int c = blk * NC + gi;
    const bool has = c < a.ncells;
    const int64_t base = (int64_t)c * bin;
    // the cell's loads are issued together: count, the first SMALL tag slots and the
    // leader's NTC state
    uint32_t n_all = has ? a.count_d[c] : 0u;
    uint32_t vl[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t k = (uint32_t)(gl + G * r);
        vl[r] = (has && k < bin) ? a.tag[base + k] : 0xFFFFFFFFu;
    }
    uint32_t nb0 = 0;
    Real cm0 = (Real)0, rem0 = (Real)0;
    if (has && gl == 0) {
        nb0 = a.nbar_sum[c];
        cm0 = a.crmax[c];
        rem0 = a.rem[c];
    }
    if (n_all > bin) n_all = bin;
    // the cells' regions of the block pool (exclusive scan of the counts); if they do not
    // fit, the cells take the whole pool one after another
    if (gl == 0) s_n[gi] = n_all;
    __syncthreads();
    if (w == 0) {
        const uint32_t x = s_n[lane];
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= (unsigned)o) inc += t;
        }
        s_off[lane] = inc - x;
        if (lane == 31) s_fits = inc <= pool ? 1u : 0u;
    }
    __syncthreads();
    const bool fits = s_fits != 0u;
    const int rounds = fits ? 1 : NC;
    for (int round = 0; round < rounds; ++round) {
        const bool act = fits || gi == round;
        const bool has_r = has && act;
        const uint32_t n = act ? n_all : 0u;
        const uint32_t poff = fits ? s_off[gi] : 0u;
        Real* vx = pv + poff;
        Real* vy = pv + pool + poff;
        Real* vz = pv + 2 * pool + poff;
        uint32_t* st = pst + poff;
        // A. stable order (ascending origin slot) and gather. Cells of up to SMALL particles
        // are sorted by their group with R keys per lane. A warp that holds a cell of up to
        // 2 SMALL puts the tags of its cells in their shared-memory tag slots and sorts them
        // two cells at a time, 2 G lanes with R keys each per cell. Larger cells are ranked
        // in shared memory.
        {
            if (__any_sync(kFull, n > (uint32_t)SMALL && n <= (uint32_t)(2 * SMALL))) {
                const bool in2 = n <= (uint32_t)(2 * SMALL);
                const uint32_t nn = in2 ? n : 0u;
                uint32_t hi[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t k = (uint32_t)(SMALL + gl + G * r);
                    hi[r] = k < nn ? a.tag[base + k] : 0u;
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t k = (uint32_t)(gl + G * r);
                    if (k < nn) st[k] = vl[r];
                    if (k + SMALL < nn) st[k + SMALL] = hi[r];
                }
                __syncwarp();
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    const int g2 = 2 * h + (int)(lane >> 4);  // the group whose cell this half sorts
                    const int l2 = (int)(lane & 15u);
                    const uint32_t n2 = __shfl_sync(kFull, nn, g2 * G);
                    uint32_t* st2 = pst + __shfl_sync(kFull, poff, g2 * G);
                    uint32_t v[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const uint32_t k = (uint32_t)(l2 + 2 * G * r);
                        v[r] = k < n2 ? st2[k] : 0xFFFFFFFFu;
                    }
                    __syncwarp();
                    bitonic_blocked<2 * G, R, R>(v);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const uint32_t pos = (uint32_t)(r + R * l2);
                        if (pos < n2) st2[pos] = v[r];
                    }
                    __syncwarp();
                }
                if (in2) {
#pragma unroll 1
                    for (int q = 0; q < 2; ++q) {
                        uint32_t src[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const uint32_t k = (uint32_t)(SMALL * q + gl + G * r);
                            src[r] = k < n ? st[k] : 0u;
                        }
                        gather_slots<Real, G, R, Z3>(a.rec, a.dx + base, a.dy + base, a.dz + base,
                                                     SMALL * q + gl, n, src, vx, vy, vz);
                    }
                }
            } else {
                uint32_t v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t k = (uint32_t)(gl + G * r);
                    v[r] = (n <= (uint32_t)SMALL && k < n) ? vl[r] : 0xFFFFFFFFu;
                }
                bitonic_blocked<G, R, R>(v);
                blocked_to_strided<G, R, R>(v, st, n <= (uint32_t)SMALL ? n : 0u, gl);
                if (n <= (uint32_t)SMALL)
                    gather_slots<Real, G, R, Z3>(a.rec, a.dx + base, a.dy + base, a.dz + base, gl,
                                                 n, v, vx, vy, vz);
            }
            if (n > (uint32_t)(2 * SMALL))
                for (uint32_t k = gl; k < n; k += G) st[k] = a.tag[base + k];
            __syncwarp();
            if (n > (uint32_t)(2 * SMALL)) {
                // rank of each tag = number of smaller tags in the cell
                for (uint32_t k = gl; k < n; k += G) {
                    const uint32_t t = st[k];
                    uint32_t r = 0;
                    for (uint32_t m = 0; m < n; ++m) r += st[m] < t ? 1u : 0u;
                    Real px, py, ux, uy, uz, pz;
                    rec_load<Z3>(a.rec, (int64_t)t, px, py, ux, uy, uz, pz);
                    a.dx[base + r] = px;
                    a.dy[base + r] = py;
                    if constexpr (Z3) a.dz[base + r] = pz;
                    vx[r] = ux;
                    vy[r] = uy;
                    vz[r] = uz;
                }
            }
        }
        // N_cand = 1/2 N Nbar F_N (sigma c_r)_max dt / V_c + remainder (group leader)
        if (gl == 0) {
            uint32_t nsel = 0;
            if (has_r) {
                const uint32_t nb = nb0 + n;
                a.nbar_sum[c] = nb;
                a.count_s[c] = 0;  // the source half's count is not needed after the move
                nlive += n;
                if (n > 32767u) {
                    flags |= HYB_ST_CELL_OVERFLOW;  // pair indices are packed in 15 and 16 bits
                } else if (n >= 2) {
                    const Real nbar = (Real)nb / (Real)(s + 1u);
                    const Real cdt = a.coll_cell ? a.coll_cell[c] : coll_dt;
                    const Real ncand = (Real)0.5 * (Real)n * nbar * cm0 * cdt + rem0;
                    const Real fl = floor(ncand);
                    a.rem[c] = ncand - fl;
                    if (fl > (Real)16777215) {
                        nsel = 16777215u;
                        flags |= HYB_ST_CELL_OVERFLOW;
                    } else {
                        nsel = (uint32_t)fl;
                    }
                }
                ncand_tot += nsel;
            }
            s_nsel[gi] = nsel;
            s_cm[gi] = cm0;
        }
        __syncthreads();
        // B. NTC collisions. The candidates of all cells are drawn in parallel by the whole
        // block, then warp 0 applies them in order, one lane per cell. If the block's
        // candidates fit the candidate buffer they are packed (cell g at the exclusive scan
        // of the counts) and drawn in one pass; otherwise every pass draws up to KC
        // candidates per cell.
        const uint32_t my_sel = s_nsel[lane];
        uint32_t sel_inc = my_sel;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, sel_inc, o);
            if (lane >= (unsigned)o) sel_inc += t;
        }
        const uint32_t sel_total = __shfl_sync(kFull, sel_inc, 31);
        const bool packed = sel_total <= (uint32_t)(NC * KC);
        const uint32_t maxsel = __reduce_max_sync(kFull, my_sel);
        const uint32_t npass = packed ? (sel_total > 0u ? 1u : 0u) : (maxsel + KC - 1) / KC;
        const int tend = packed ? (int)sel_total : NC * KC;
        Real cm = (Real)0;
        uint32_t ncoll = 0;
        Real* gvx = nullptr;
        Real* gvy = nullptr;
        Real* gvz = nullptr;
        if (w == 0) {
            cm = s_cm[lane];
            const uint32_t go = fits ? s_off[lane] : 0u;
            gvx = pv + go;
            gvy = pv + pool + go;
            gvz = pv + 2 * pool + go;
        }
        for (uint32_t pass = 0; pass < npass; ++pass) {
            const uint32_t k0 = pass * (uint32_t)KC;
            for (int tb = w * 32; tb < tend; tb += WARPS * 32) {  // warp-uniform trip count
                const int t = tb + (int)lane;
                int g;
                uint32_t k;
                bool valid;
                if (packed) {
                    // the cell whose range holds slot t: the number of cells whose inclusive
                    // count is <= t
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const uint32_t v = __shfl_sync(kFull, sel_inc, lo + step - 1);
                        if (v <= (uint32_t)t) lo += step;
                    }
                    g = lo;
                    const uint32_t ginc = __shfl_sync(kFull, sel_inc, g);
                    const uint32_t gsel = __shfl_sync(kFull, my_sel, g);
                    k = (uint32_t)t - (ginc - gsel);
                    valid = t < tend;
                } else {
                    g = t / KC;
                    k = k0 + (uint32_t)(t % KC);
                    valid = t < tend && k < s_nsel[g];
                }
                if (valid) {
                    const uint32_t cg = (uint32_t)(blk * NC + g);
                    const uint32_t ng = s_n[g];
                    const uint4 r = draw(a.seed, cg, s, TAG_NTC_PAIR, k, 0);
                    const uint32_t ci = uindex(r.x, ng);
                    uint32_t cj = uindex(r.y, ng - 1u);
                    if (cj >= ci) cj += 1u;
                    Real nx = (Real)0, ny = (Real)0, nz = (Real)0;
                    const int ok = unit_vector(a.seed, cg, s, k, nx, ny, nz);
                    c_ij[t] = ci | (cj << 15) | (ok ? 0u : 0x80000000u);
                    c_R[t] = (Real)u01f(r.z);
                    c_nx[t] = nx;
                    c_ny[t] = ny;
                    c_nz[t] = nz;
                }
            }
            __syncthreads();
            if (w == 0) {
                // the candidates of this pass for the lane's cell; the particles of the next
                // candidate are loaded before this one is applied, and taken from registers
                // where this one changes them
                const int kend = packed ? (int)my_sel
                                        : (my_sel > k0 ? (int)min(my_sel - k0, (uint32_t)KC) : 0);
                const int t0 = packed ? (int)(sel_inc - my_sel) : (int)lane * KC;
                uint32_t ijn = 0;
                Real nax = 0, nay = 0, naz = 0, nbx = 0, nby = 0, nbz = 0;
                if (kend > 0) {
                    ijn = c_ij[t0];
                    const uint32_t i = ijn & 0x7FFFu, j = (ijn >> 15) & 0xFFFFu;
                    nax = gvx[i], nay = gvy[i], naz = gvz[i];
                    nbx = gvx[j], nby = gvy[j], nbz = gvz[j];
                }
#pragma unroll 1
                for (int kk = 0; kk < kend; ++kk) {
                    const int t = t0 + kk;
                    const uint32_t ij = ijn;
                    const uint32_t i = ij & 0x7FFFu, j = (ij >> 15) & 0xFFFFu;
                    const Real ax = nax, ay = nay, az = naz;
                    const Real bx = nbx, by = nby, bz = nbz;
                    uint32_t in_ = 0xFFFFFFFFu, jn = 0xFFFFFFFFu;
                    if (kk + 1 < kend) {
                        ijn = c_ij[t + 1];
                        in_ = ijn & 0x7FFFu;
                        jn = (ijn >> 15) & 0xFFFFu;
                        nax = gvx[in_], nay = gvy[in_], naz = gvz[in_];
                        nbx = gvx[jn], nby = gvy[jn], nbz = gvz[jn];
                    }
                    const Real ddx = ax - bx, ddy = ay - by, ddz = az - bz;
                    const Real cr = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                    if (cr > cm) cm = cr;
                    if (cr > c_R[t] * cm) {
                        if (ij & 0x80000000u) {
                            flags |= HYB_ST_SCATTER_CAP;
                        } else {
                            const Real cx = (ax + bx) * (Real)0.5;
                            const Real cy = (ay + by) * (Real)0.5;
                            const Real cz = (az + bz) * (Real)0.5;
                            const Real h = cr * (Real)0.5;
                            const Real hx = h * c_nx[t], hy = h * c_ny[t], hz = h * c_nz[t];
                            const Real pix = cx + hx, piy = cy + hy, piz = cz + hz;
                            const Real pjx = cx - hx, pjy = cy - hy, pjz = cz - hz;
                            gvx[i] = pix;
                            gvy[i] = piy;
                            gvz[i] = piz;
                            gvx[j] = pjx;
                            gvy[j] = pjy;
                            gvz[j] = pjz;
                            ncoll += 1;
                            if (in_ == i) nax = pix, nay = piy, naz = piz;
                            if (in_ == j) nax = pjx, nay = pjy, naz = pjz;
                            if (jn == i) nbx = pix, nby = piy, nbz = piz;
                            if (jn == j) nbx = pjx, nby = pjy, nbz = pjz;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (w == 0) {
            const int cl = blk * NC + (int)lane;
            if (cl < a.ncells && (fits || (int)lane == round)) a.crmax[cl] = cm;
            ncoll_tot += ncoll;
        }
        // C. write-out and moment sums (group lanes over the cell's particles)
        Real mo[kMoments];
#pragma unroll
        for (int q = 0; q < kMoments; ++q) mo[q] = (Real)0;
        for (uint32_t k = gl; k < n; k += G) {
            const Real ux = vx[k], uy = vy[k], uz = vz[k];
            a.dvx[base + k] = ux;
            a.dvy[base + k] = uy;
            a.dvz[base + k] = uz;
            if (do_sample) {
                // the sums are compared with a tolerance, so they use fused multiply-adds
                // (this file is otherwise compiled without contraction); mo[0] is the count
                const Real xx = ux * ux, yy = uy * uy, zz = uz * uz, xy = ux * uy;
                mo[1] += ux; mo[2] += uy; mo[3] += uz;
                mo[4] += xx; mo[5] = fma(ux, uy, mo[5]); mo[6] = fma(ux, uz, mo[6]);
                mo[7] += yy; mo[8] = fma(uy, uz, mo[8]); mo[9] += zz;
                mo[10] = fma(xx, ux, mo[10]); mo[11] = fma(xx, uy, mo[11]);
                mo[12] = fma(xx, uz, mo[12]); mo[13] = fma(yy, ux, mo[13]);
                mo[14] = fma(xy, uz, mo[14]); mo[15] = fma(zz, ux, mo[15]);
                mo[16] = fma(yy, uy, mo[16]); mo[17] = fma(yy, uz, mo[17]);
                mo[18] = fma(zz, uy, mo[18]); mo[19] = fma(zz, uz, mo[19]);
            }
        }
        if (do_sample) {
            // halving exchange over the group: lane gl ends with the totals of moments
            // 3 gl, 3 gl + 1, 3 gl + 2
            Real t[24];
#pragma unroll
            for (int q = 0; q < 24; ++q) t[q] = q < kMoments ? mo[q] : (Real)0;
#pragma unroll
            for (int o = G / 2, len = 12; o >= 1; o >>= 1, len >>= 1) {
                const bool hi = (gl & o) != 0;
#pragma unroll
                for (int q = 0; q < len; ++q) {
                    const Real send = hi ? t[q] : t[q + len];
                    const Real keep = hi ? t[q + len] : t[q];
                    t[q] = keep + __shfl_xor_sync(kFull, send, o);
                }
            }
            if (gl == 0) t[0] = (Real)n;  // the particle count, moment 0
            if (has_r) {
                // one FP64 addition per sum, done in L2 (each sum has one writer per step)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int mq = 3 * gl + q;
                    if (mq < kMoments) atomicAdd(&a.acc[(size_t)c * kMoments + mq], widen(t[q]));
                }
            }
        }
        __syncthreads();  // the pool is reused by the next round
    }
    // event counters: per block, one atomic per counter
    ncand_tot = __reduce_add_sync(kFull, (unsigned)ncand_tot);
    ncoll_tot = __reduce_add_sync(kFull, (unsigned)ncoll_tot);
    nlive = __reduce_add_sync(kFull, nlive);
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0) {
        s_cnt[w][0] = ncand_tot;
        s_cnt[w][1] = ncoll_tot;
        s_live[w] = nlive;
        s_flags[w] = flags;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long c0 = 0, c1 = 0;
        uint32_t nl = 0, fl = 0;
        for (int v = 0; v < WARPS; ++v) {
            c0 += s_cnt[v][0];
            c1 += s_cnt[v][1];
            nl += s_live[v];
            fl |= s_flags[v];
        }
        if (c0) atomicAdd(&a.counters[HYB_C_CANDIDATES], c0);
        if (c1) atomicAdd(&a.counters[HYB_C_COLLISIONS], c1);
        if (nl) atomicAdd(&a.ctrl[CTRL_NTOT], nl);
        if (fl) atomicOr(&a.ctrl[CTRL_STATUS], fl);
        // the last block to finish advances the step and sample counters (every block has
        // read the step by now; nothing written by other blocks is read here, so no fence
        // is needed before the ticket)
        const unsigned ticket = atomicAdd(&a.ctrl[CTRL_TICKET], 1u);
        if (ticket == nblk - 1) {
            __threadfence();
            if (do_sample) a.ctrl[CTRL_NSAMPLES] += 1;
            a.ctrl[CTRL_STEP] = s + 1;
            a.ctrl[CTRL_TICKET] = 0;
        }
    }
}

template <typename Real, bool BATCH, bool Z3 = false>
__global__ void __launch_bounds__(kCollideWarps * 32, CollideCfg<Real>::MINB)
    k_collide(Launch<DsmcArgs<Real>> L, uint32_t pool) {
    pdl_begin();
    if constexpr (BATCH) {
        const int r = replica_of(L.pre, L.nrep, (int64_t)blockIdx.x);
        collide_block<Real, Z3>(L.tab[r], pool, (int)(blockIdx.x - L.pre[r]),
                                (int)(L.pre[r + 1] - L.pre[r]));
    } else {
        collide_block<Real, Z3>(L.one, pool, (int)blockIdx.x, (int)gridDim.x);
    }
}

template <typename Real>
DsmcArgs<Real> make_args(Ctx& c) {
    DsmcArgs<Real> a{};
    const int h = c.cur_p, o = c.cur_p ^ 1;
    a.sx = (const Real*)c.st.px[h];
    a.sy = (const Real*)c.st.py[h];
    a.svx = (const Real*)c.st.pvx[h];
    a.svy = (const Real*)c.st.pvy[h];
    a.svz = (const Real*)c.st.pvz[h];
    a.rec = (Real*)c.st.moved;
    a.dx = (Real*)c.st.px[o];
    a.dy = (Real*)c.st.py[o];
    a.dvx = (Real*)c.st.pvx[o];
    a.dvy = (Real*)c.st.pvy[o];
    a.dvz = (Real*)c.st.pvz[o];
    a.tag = c.st.tag;
    a.count_s = c.st.count[h];
    a.count_d = c.st.count[o];
    a.crmax = (Real*)c.st.crmax;
    a.rem = (Real*)c.st.rem;
    a.nbar_sum = c.st.nbar_sum;
    a.acc = c.st.acc;
    a.ctrl = c.st.ctrl;
    a.counters = c.st.counters;
    a.ncx = c.p.ncx;
    a.ncy = c.p.ncy;
    a.ncells = (int32_t)c.d.ncells;
    a.bin = c.d.bin;
    a.sample_every = c.p.sample_every;
    a.ppc = c.p.ppc;
    a.dt = c.d.dt;
    a.g_step = c.d.g_step;
    a.coll_dt = c.d.coll_dt;
    a.dt_r = (Real)c.d.dt;
    a.g_r = (Real)c.d.g_step;
    a.coll_r = (Real)c.d.coll_dt;
    a.coll_cell = (const Real*)c.st.coll_cell;
    a.sz = (const Real*)c.st.pz[h];
    a.dz = (Real*)c.st.pz[o];
    a.ncz = c.p.ncz >= 2 ? c.p.ncz : 0;
    a.crmax_init = c.p.crmax_init;
    a.seed = c.p.seed;
    return a;
}

int grid_for(const Ctx& c, int64_t work, int threads, int per_sm) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)c.num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename Real>
cudaError_t init_impl(Ctx& c) {
    // the initial particles go to half 0: arguments built with half 1 as the source
    c.cur_p = 1;
    DsmcArgs<Real> a = make_args<Real>(c);
    c.cur_p = 0;
    const int64_t n = c.d.ncells * c.p.ppc;
    k_init_particles<Real><<<grid_for(c, n, 256, 16), 256, 0, c.stream>>>(a);
    k_init_cells<Real><<<grid_for(c, c.d.ncells, 256, 16), 256, 0, c.stream>>>(a);
    return cudaGetLastError();
}

template <typename Real, bool Z3>
cudaError_t step_impl(Ctx& c) {
    DsmcArgs<Real> a = make_args<Real>(c);
    prof_begin(c, K_MOVE);
    // one source cell per warp (the hardware schedules the blocks as resources free up)
    Launch<DsmcArgs<Real>> L{};
    L.one = a;
    L.total = c.d.ncells;
    cudaError_t e = launch_pdl(k_move<Real, false, Z3>, dim3(grid_for(c, c.d.ncells * 32, 256, 64)),
                               dim3(256), 0, c.stream, L);
    if (e != cudaSuccess) return e;
    prof_end(c, K_MOVE);
    // shared memory: a pool of slots for the block's cells (3 Real + 1 u32 each), room for
    // 1.5 ppc per cell on average and at least one full bin, then one pass of NTC candidates
    constexpr int NC = kCollideWarps * (32 / kGroup);
    uint32_t pool = (uint32_t)(((int64_t)NC * c.p.ppc * 3 / 2 + 31) / 32 * 32);
    if (pool < (uint32_t)c.d.bin) pool = (uint32_t)c.d.bin;
    const size_t smem = (size_t)pool * (3 * sizeof(Real) + 4) +
                        (size_t)NC * kChainSteps * (4 + 4 * sizeof(Real));
    // (dynamic and static shared memory together may exceed the default 48 KB)
    e = cudaFuncSetAttribute(k_collide<Real, false, Z3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((c.d.ncells + NC - 1) / NC);
    prof_begin(c, K_COLLIDE);
    L.total = grid;
    e = launch_pdl(k_collide<Real, false, Z3>, dim3(grid), dim3(kCollideWarps * 32), smem, c.stream, L,
                   pool);
    if (e != cudaSuccess) return e;
    prof_end(c, K_COLLIDE);
    return cudaGetLastError();
}

__global__ void k_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]),
                               (uint32_t)seed, (uint32_t)(seed >> 32));
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

}  // namespace

cudaError_t launch_lbm_init(Ctx& c);

cudaError_t launch_init(Ctx& c) {
    cudaError_t e = (c.p.real_bytes == 4) ? init_impl<float>(c) : init_impl<double>(c);
    if (e != cudaSuccess) return e;
    return launch_lbm_init(c);
}

cudaError_t launch_dsmc_step(Ctx& c) {
    if (c.p.ncz >= 2) return (c.p.real_bytes == 4) ? step_impl<float, true>(c) : step_impl<double, true>(c);
    return (c.p.real_bytes == 4) ? step_impl<float, false>(c) : step_impl<double, false>(c);
}

size_t dsmc_args_bytes(int real_bytes) {
    return real_bytes == 4 ? sizeof(DsmcArgs<float>) : sizeof(DsmcArgs<double>);
}

void dsmc_args_fill(Ctx& c, int cur_p, void* out) {
    const int save = c.cur_p;
    c.cur_p = cur_p;
    if (c.p.real_bytes == 4) {
        const DsmcArgs<float> a = make_args<float>(c);
        std::memcpy(out, &a, sizeof(a));
    } else {
        const DsmcArgs<double> a = make_args<double>(c);
        std::memcpy(out, &a, sizeof(a));
    }
    c.cur_p = save;
}

uint32_t collide_pool(const Ctx& c) {
    constexpr int NC = kCollideWarps * (32 / kGroup);
    uint32_t pool = (uint32_t)(((int64_t)NC * c.p.ppc * 3 / 2 + 31) / 32 * 32);
    if (pool < (uint32_t)c.d.bin) pool = (uint32_t)c.d.bin;
    return pool;
}

namespace {

template <typename Real>
cudaError_t batch_move_impl(BatchDev& b, int cur_p) {
    Launch<DsmcArgs<Real>> L{};
    L.tab = (const DsmcArgs<Real>*)b.dsmc[cur_p];
    L.pre = b.pre_cells;
    L.nrep = b.nrep;
    L.total = b.tot_cells;
    const int64_t blocks = (b.tot_cells * 32 + b.move_block - 1) / b.move_block;
    return launch_pdl(k_move<Real, true>, dim3((unsigned)blocks), dim3(b.move_block), 0, b.stream, L);
}

template <typename Real>
cudaError_t batch_collide_impl(BatchDev& b, int cur_p) {
    constexpr int NC = kCollideWarps * (32 / kGroup);
    Launch<DsmcArgs<Real>> L{};
    L.tab = (const DsmcArgs<Real>*)b.dsmc[cur_p];
    L.pre = b.pre_blocks;
    L.nrep = b.nrep;
    L.total = b.tot_blocks;
    const size_t smem = (size_t)b.pool * (3 * sizeof(Real) + 4) + (size_t)NC * kChainSteps * (4 + 4 * sizeof(Real));
    cudaError_t e = cudaFuncSetAttribute(k_collide<Real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_collide<Real, true>, dim3((unsigned)b.tot_blocks), dim3(kCollideWarps * 32), smem,
                      b.stream, L, b.pool);
}

}  // namespace

cudaError_t launch_batch_move(BatchDev& b, int cur_p) {
    return b.real_bytes == 4 ? batch_move_impl<float>(b, cur_p) : batch_move_impl<double>(b, cur_p);
}

cudaError_t launch_batch_collide(BatchDev& b, int cur_p) {
    return b.real_bytes == 4 ? batch_collide_impl<float>(b, cur_p) : batch_collide_impl<double>(b, cur_p);
}

cudaError_t launch_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n,
                                cudaStream_t s) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_debug_philox<<<(int)g, 256, 0, s>>>(ctr, seed, out, n);
    return cudaGetLastError();
}

}  // namespace hyb
