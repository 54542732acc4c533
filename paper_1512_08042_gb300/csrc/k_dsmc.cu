// DSMC kernels: initialisation, the move with diffuse isothermal walls and binning by cell,
// and the per-cell stable ordering, no-time-counter hard-sphere collisions and
// Hermite-moment sampling.
//
// Particles live in per-cell bins of `bin` slots (cell c owns slots [c bin, (c+1) bin) of
// each state array, count[c] in use) and ping-pong between two halves. A DSMC step (the NTC
// order of Bird that the paper uses in Sec. 5: move, index, collide, sample) from the sorted
// particles of half p takes two passes:
//   k_move     one warp per source cell: body-force kick, free flight, diffuse wall
//              re-emission (Sec. 3.1), periodic wrap, new cell; the moved particle and its
//              order key (its displacement's neighbour offset, then its rank in the old cell;
//              see order_key) are appended to the bin of its new cell in half p^1 by a
//              warp-aggregated atomic.
//   k_collide  32 consecutive cells per block, a group of 8 lanes per cell: each arrival's
//              rank by key comes from a bitmap of the cell's keys with prefix counts, each
//              arrival is placed at its rank in a shared-memory pool, the NTC candidates of
//              all 32 cells are drawn by the whole
//              block and applied by one warp with a lane per cell (Eq. collisionnumber), the
//              sums 1, v, vv, vvv are added to the FP64 cumulative sums of the cell (Sec. 2.1,
//              Fig. 1) and the sorted cell is written back in place.
//   k_step_end one thread per context after each collide pass: publishes the particle count
//              and advances the step and sample counters.
// Several steps in one call fuse the collide of step s with the move of step s + 1: the
// fused pass collides and samples a cell as above and then moves its particles straight from
// the pool into the bins of the other half, so a particle's state is read and written once
// per step. Cells that the step's LB2DSMC regenerates are written back in place instead.
// This file is compiled without FMA contraction so that positions, cell keys, pair choices
// and post-collision velocities are the IEEE float (or double) results of the written
// expressions.
#include <cstring>

#include "dsmc_move.cuh"

namespace hyb {

namespace {

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
        const uint32_t cl = (uint32_t)(s / a.ppc), k = (uint32_t)(s % a.ppc);
        const int ix = (int)(cl % (uint32_t)a.ncx);
        const int iy = a.y0 + (int)((cl / (uint32_t)a.ncx) % (uint32_t)a.ncy);  // the channel's row
        const int64_t slot = (int64_t)cl * a.bin + k;
        const uint32_t c = global_cell(cl, a.ncx, a.ncy, a.y0, a.ncy_g);  // key of the draws
        const uint4 rp = draw(a.seed, c, 0, TAG_INIT_POS, k, 0);
        const Real px = (Real)ix + (Real)u01f(rp.x);
        const Real py = (Real)iy + (Real)u01f(rp.y);
        const Real pz = a.ncz ? (Real)(cl / ((uint32_t)a.ncx * (uint32_t)a.ncy)) + (Real)u01f(rp.z)
                              : (Real)0;
        const uint4 rv = draw(a.seed, c, 0, TAG_INIT_VEL, k, 0);
        Real n0, n1, n2, n3;
        gauss_pair<Real>(rv.x, rv.y, n0, n1);
        gauss_pair<Real>(rv.z, rv.w, n2, n3);
        rec_put(a.drec, slot, px, py, pz, n0, n1, n2, 0u);
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

// ---------------------------------------------------------------------------------------
// Move (kick, drift, walls, wrap) of the sorted particles of half p into the bins of p^1.

template <typename Real>
__device__ __forceinline__ MoveCtx<Real> move_ctx(const DsmcArgs<Real>& a) {
    MoveCtx<Real> m;
    m.H = (Real)a.ncx;
    m.L = (Real)a.ncy_g;
    m.Lz = (Real)(a.ncz ? a.ncz : 1);
    m.dt = a.dt_r;
    m.g = a.g_r;
    m.ncx = a.ncx;
    m.ncy = a.ncy_g;
    m.ncz = a.ncz;
    m.y0 = a.y0;
    m.nly = a.ncy;
    m.bin = (uint32_t)a.bin;
    m.seed = a.seed;
    return m;
}

template <typename Real>
__device__ __forceinline__ Half<Real> half_s(const DsmcArgs<Real>& a) {
    return Half<Real>{a.srec, a.count_s};
}
template <typename Real>
__device__ __forceinline__ Half<Real> half_d(const DsmcArgs<Real>& a) {
    return Half<Real>{a.drec, a.count_d};
}

// One source cell, by one warp; 64 particles of the cell at a time, two per lane, with the
// loads, flights and binning atomics of both in flight together.
template <typename Real, bool Z3>
__device__ __forceinline__ void move_cell(const DsmcArgs<Real>& a, int c, unsigned lane) {
    const uint32_t s = a.ctrl[CTRL_STEP];
    const MoveCtx<Real> m = move_ctx(a);
    const uint32_t bin = (uint32_t)a.bin;
    // the halves do not overlap: loads of the next records need not wait for earlier stores
    const Real* __restrict__ src = a.srec;
    const Half<Real> dst = half_d(a);
    uint32_t hits = 0, caps = 0, lost = 0;
    uint32_t n = a.count_s[c];
    __syncwarp();
    if (lane == 0) a.count_s[c] = 0;  // half p is consumed; its counts start the next arrivals
    if (n > bin) n = bin;
    const int64_t base = (int64_t)c * bin;
    // the channel's cell: the key of the wall draws and of the order keys
    const Origin org = origin_of(m, global_cell((uint32_t)c, a.ncx, a.ncy, a.y0, a.ncy_g));
    for (uint32_t k0 = 0; k0 == 0 || k0 < n; k0 += 64) {
        const uint32_t k1 = k0 + lane, k2 = k1 + 32;
        const bool act1 = k1 < n, act2 = k2 < n;
        Real p1[6] = {0, 0, 0, 0, 0, 0}, p2[6] = {0, 0, 0, 0, 0, 0};  // x y z vx vy vz
        uint32_t t1, t2;
        // the loads need only the bin size, not the count, so they travel with it
        if (k1 < bin) rec_get(src, base + k1, p1[0], p1[1], p1[2], p1[3], p1[4], p1[5], t1);
        if (k2 < bin) rec_get(src, base + k2, p2[0], p2[1], p2[2], p2[3], p2[4], p2[5], t2);
        uint32_t key1 = 0, key2 = 0, ok1 = 0, ok2 = 0;
        int dir1 = -1, dir2 = -1;
        if (act1)
            key1 = move_particle<Real, Z3>(m, org, k1, s, p1[0], p1[1], p1[2], p1[3], p1[4], p1[5], hits,
                                           caps, dir1, ok1);
        if (act2)
            key2 = move_particle<Real, Z3>(m, org, k2, s, p2[0], p2[1], p2[2], p2[3], p2[4], p2[5], hits,
                                           caps, dir2, ok2);
        const bool loc1 = act1 && dir1 < 0, loc2 = act2 && dir2 < 0;
        uint32_t arr1, arr2;
        bin_arrival2(dst.count, key1, loc1, key2, loc2, lane, arr1, arr2);
        if (loc1) {
            if (arr1 < bin)
                put_particle<Real, Z3>(dst, (int64_t)key1 * bin + arr1, ok1, p1[0], p1[1], p1[2], p1[3],
                                       p1[4], p1[5]);
            else
                lost += 1;
        } else if (act1) {
            send_particle<Real, Z3>(a.xrec, a.xkey, a.xcount, a.xcap, dir1, key1, ok1, p1[0], p1[1],
                                    p1[2], p1[3], p1[4], p1[5], lost);
        }
        if (loc2) {
            if (arr2 < bin)
                put_particle<Real, Z3>(dst, (int64_t)key2 * bin + arr2, ok2, p2[0], p2[1], p2[2], p2[3],
                                       p2[4], p2[5]);
            else
                lost += 1;
        } else if (act2) {
            send_particle<Real, Z3>(a.xrec, a.xkey, a.xcount, a.xcap, dir2, key2, ok2, p2[0], p2[1],
                                    p2[2], p2[3], p2[4], p2[5], lost);
        }
    }
    move_events(a.counters, a.ctrl, hits, caps, lost, lane);
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
// Collide: a group of G lanes per cell, 32 / G cells per warp. Every instruction of the
// serial NTC chain then advances 32 / G cells at once. All loops that contain shuffles have
// warp-uniform trip counts (groups whose cell has less work are masked), so every shuffle is
// executed by the full warp.
constexpr int kGroup = 8;

// A collide block has W warps for 4 W cells (W = 8: 32 cells, the default; W = 4: 16 cells,
// twice the blocks per SM); its launch bounds keep 80 registers (FP32) or 128 (FP64).
constexpr int kCollideWarps = 8;
template <typename Real, int W>
struct CollideCfg {
    static constexpr int MINB = (sizeof(Real) == 4 ? 3 : 2) * 8 / W;  // resident blocks per SM
};
constexpr int kChainSteps = 24;   // candidates per cell drawn per pass of the NTC phase
enum CollideMode : int { MODE_COLLIDE = 0, MODE_FUSED = 1 };

// Real arrays of the shared-memory pool per slot: vx, vy, vz, x, y (, z)
template <bool Z3>
__host__ __device__ constexpr int pool_reals() {
    return Z3 ? 6 : 5;
}

// Words of a cell's order-key bitmap: one bit per key below W bin, W = 9 neighbour offsets in
// 2D and 27 in 3D (bin is a multiple of 32).
template <bool Z3>
__host__ __device__ constexpr int bitmap_words(uint32_t bin) {
    return (Z3 ? 27 : 9) * (int)(bin / 32u);
}
// Keys of farther-displaced particles a cell lists for their ranks (more are counted in full).
constexpr int kFarList = 8;

// Adds a particle's velocity moments to a lane's partial sums: u, the six distinct products
// u_i u_j and the ten distinct u_i u_j u_k, in the order of the sampled sums (mo[0], the count,
// is set after the reduction). The sums are compared with a tolerance, so they use fused
// multiply-adds (this file is otherwise compiled without contraction).
template <typename Real>
__device__ __forceinline__ void add_moments(Real (&mo)[kMoments], Real ux, Real uy, Real uz) {
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

// The block of 32 consecutive cells `blk` (of nblk) of one context: the arrivals of half
// p^1 (d*) are put in stable order, collided and sampled; MODE_COLLIDE writes them back in
// place, MODE_FUSED moves them on (step s + 1) into the bins of half p (s*), except cells
// marked in a.coupled, which are written back in place for LB2DSMC.
template <typename Real, bool Z3, int MODE, int W>
__device__ __forceinline__ void collide_block(const DsmcArgs<Real>& a, uint32_t pool, int blk) {
    constexpr int G = kGroup;
    constexpr int CPW = 32 / G;           // cells per warp in phases A and C
    constexpr int WARPS = W;
    constexpr int NC = WARPS * CPW;       // cells per block (one chain lane each in phase B)
    constexpr int SMALL = 64;             // keys of the first SMALL slots loaded with the count
    constexpr int R = SMALL / G;
    constexpr int KC = kChainSteps;       // candidates per cell drawn per pass of phase B
    constexpr int NR = pool_reals<Z3>();
    constexpr int SJ = 2;                 // arrivals per lane whose loads are in flight together
    static_assert(NC <= 32, "phase B runs one lane per cell of the block in one warp");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // per cell of the block, by phase B's lanes (lanes past NC are empty cells)
    __shared__ uint32_t s_n[32], s_off[32], s_nsel[32];
    __shared__ Real s_cm[32];
    if (NC < 32 && threadIdx.x >= NC && threadIdx.x < 32) {
        s_n[threadIdx.x] = 0u;
        s_nsel[threadIdx.x] = 0u;
        s_cm[threadIdx.x] = (Real)0;
    }
    __shared__ uint32_t s_fits;
    __shared__ unsigned long long s_cnt[WARPS][2];
    __shared__ uint32_t s_live[WARPS], s_flags[WARPS];
    __shared__ __align__(16) double s_acc[NC][kMoments];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int grp = (int)lane / G, gl = (int)lane % G;
    const int gi = w * CPW + grp;  // the group's cell within the block
    const uint32_t bin = (uint32_t)a.bin;
    // shared memory: the block's pool of vx, vy, vz, x, y (, z) (Real), `pool` slots each, then the candidates of one pass of phase B, in the same space as the cells'
    // key bitmaps of phase A (BW words and BW prefix bytes per cell)
    Real* pv = reinterpret_cast<Real*>(smem_raw);
    uint32_t* c_ij = reinterpret_cast<uint32_t*>(pv + NR * (size_t)pool);
    const int BW = bitmap_words<Z3>(bin);
    const int CW = (BW + G - 1) / G;
    const uint32_t lim = (uint32_t)BW * 32u;
    uint32_t* s_bm = c_ij;
    uint32_t* s_fl = s_bm + NC * BW;
    uint8_t* s_pf = reinterpret_cast<uint8_t*>(s_fl + NC * (kFarList + 1));
    Real* c_R = reinterpret_cast<Real*>(c_ij + NC * KC);
    Real* c_nx = c_R + NC * KC;
    Real* c_ny = c_nx + NC * KC;
    Real* c_nz = c_ny + NC * KC;
    const uint32_t s = a.ctrl[CTRL_STEP];
    const bool do_sample = (s % (uint32_t)a.sample_every) == 0u;
    const Real coll_dt = a.coll_r;
    unsigned long long ncand_tot = 0, ncoll_tot = 0;
    uint32_t flags = 0, nlive = 0;
    uint32_t hits = 0, caps = 0, lost = 0;

    const int c = blk * NC + gi;
    const bool has = c < a.ncells;
    const int64_t base = (int64_t)c * bin;
    // the channel's cell: the key of the random streams and of the stable order
    const uint32_t gc = global_cell((uint32_t)c, a.ncx, a.ncy, a.y0, a.ncy_g);
    const Real* __restrict__ drec = a.drec;
    // the cell's loads are issued together: count, the first SMALL keys and the leader's NTC
    // state
    uint32_t n_all = has ? a.count_d[c] : 0u;
    // the cell's FP64 sums, copied to shared memory while the block works (10 x 16 bytes)
    if (has && do_sample)
        for (int j = gl; j < 2 * kMoments / 4; j += G)
            cp_async16(&s_acc[gi][2 * j], &a.acc[(size_t)c * kMoments + 2 * j]);
    cp_async_commit();
    uint32_t vl[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t k = (uint32_t)(gl + G * r);
        vl[r] = (has && k < bin) ? rec_tag(drec, base + k) : 0xFFFFFFFFu;
    }
    uint32_t nb0 = 0;
    Real cm0 = (Real)0, rem0 = (Real)0;
    if (has && gl == 0) {
        nb0 = a.nbar_sum[c];
        cm0 = a.crmax[c];
        rem0 = a.rem[c];
    }
    const bool moving = MODE == MODE_FUSED && has && !(a.coupled && a.coupled[c]);
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
        Real* qx = pv + 3 * pool + poff;
        Real* qy = pv + 4 * pool + poff;
        Real* qz = pv + 5 * (size_t)pool + poff;  // 3D only
        // A. stable order: every arrival's rank among the cell's arrivals by order key. A key
        // below W bin (a particle from a neighbouring cell) sets bit `key` of the cell's
        // bitmap, and its rank is the number of set bits below it: the count before its word
        // (a prefix over the words, kept modulo 256: a queried word holds its own bit, so
        // the count is below bin) plus those below it within the word. Larger keys follow
        // all of these, each ranked by counting the larger keys below it (from a list of the
        // cell's larger keys while they are few, else from the records).
        {
            uint32_t* bm = s_bm + gi * BW;
            uint8_t* pf = s_pf + gi * BW;
            uint32_t* fl = s_fl + gi * (kFarList + 1);  // count, then the first kFarList keys
            for (int q = gl; q < BW; q += G) bm[q] = 0u;
            if (gl == 0) fl[0] = 0u;
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t k = (uint32_t)(gl + G * r);
                if (k < n) {
                    const uint32_t t = vl[r];
                    if (t < lim) {
                        atomicOr(&bm[t >> 5], 1u << (t & 31u));
                    } else {
                        const uint32_t j = atomicAdd(&fl[0], 1u);
                        if (j < (uint32_t)kFarList) fl[1 + j] = t;
                    }
                }
            }
            for (uint32_t k = SMALL + gl; k < n; k += G) {
                const uint32_t t = rec_tag(drec, base + k);
                if (t < lim) {
                    atomicOr(&bm[t >> 5], 1u << (t & 31u));
                } else {
                    const uint32_t j = atomicAdd(&fl[0], 1u);
                    if (j < (uint32_t)kFarList) fl[1 + j] = t;
                }
            }
            __syncwarp();
            // the prefix counts: lane gl owns words [gl CW, gl CW + CW)
            const int q0 = gl * CW, q1 = min(q0 + CW, BW);
            uint32_t tot = 0;
            for (int q = q0; q < q1; ++q) tot += (uint32_t)__popc(bm[q]);
            uint32_t inc = tot;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, inc, o, G);
                if (gl >= o) inc += t;
            }
            uint32_t run = inc - tot;
            for (int q = q0; q < q1; ++q) {
                pf[q] = (uint8_t)run;
                run += (uint32_t)__popc(bm[q]);
            }
            const uint32_t nfar = fl[0];
            const uint32_t nnear = n - nfar;
            __syncwarp();
            // each arrival goes to the pool slot of its rank (its record carries its key); the
            // loads of a lane's arrivals can be in flight together
            for (uint32_t k0 = 0; k0 < n; k0 += SJ * G) {
                Real p[SJ][6];
                uint32_t t[SJ];
#pragma unroll
                for (int j = 0; j < SJ; ++j) {
                    const uint32_t k = k0 + (uint32_t)(gl + G * j);
                    if (k < n) rec_get(drec, base + k, p[j][3], p[j][4], p[j][5], p[j][0], p[j][1], p[j][2], t[j]);
                }
#pragma unroll
                for (int j = 0; j < SJ; ++j) {
                    const uint32_t k = k0 + (uint32_t)(gl + G * j);
                    if (k < n) {
                        uint32_t rk;
                        if (t[j] < lim) {
                            const uint32_t q = t[j] >> 5;
                            rk = (uint32_t)pf[q] + (uint32_t)__popc(bm[q] & ((1u << (t[j] & 31u)) - 1u));
                        } else if (nfar <= (uint32_t)kFarList) {
                            rk = nnear;
                            for (uint32_t m2 = 0; m2 < nfar; ++m2) rk += fl[1 + m2] < t[j] ? 1u : 0u;
                        } else {
                            rk = nnear;
                            for (uint32_t m2 = 0; m2 < n; ++m2) {
                                const uint32_t u = rec_tag(drec, base + m2);
                                rk += (u >= lim && u < t[j]) ? 1u : 0u;
                            }
                        }
                        vx[rk] = p[j][0];
                        vy[rk] = p[j][1];
                        vz[rk] = p[j][2];
                        qx[rk] = p[j][3];
                        qy[rk] = p[j][4];
                        if constexpr (Z3) qz[rk] = p[j][5];
                    }
                }
            }
        }
        // N_cand = 1/2 N Nbar F_N (sigma c_r)_max dt / V_c + remainder (group leader)
        if (gl == 0) {
            uint32_t nsel = 0;
            if (has_r) {
                const uint32_t nb = nb0 + n;
                a.nbar_sum[c] = nb;
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
                    const uint32_t cg = global_cell((uint32_t)(blk * NC + g), a.ncx, a.ncy, a.y0, a.ncy_g);
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
            if ((int)lane < NC && cl < a.ncells && (fits || (int)lane == round)) a.crmax[cl] = cm;
            ncoll_tot += ncoll;
        }
        // C. moment sums of the collided particles; the cell is written back in place in
        // stable order (the collide, and cells the step's LB2DSMC regenerates), or moved on
        // Every lane sums its particles gl, gl + G, gl + 2 G, ... in this order, whether in
        // the loop below (cells written back) or in the move (cells moved on), so that the
        // sums of a fused pass equal those of single steps bit for bit.
        Real mo[kMoments];
#pragma unroll
        for (int q = 0; q < kMoments; ++q) mo[q] = (Real)0;
        const bool back = has_r && !moving;
        const uint32_t nback = back ? n : 0u;
        for (uint32_t k = gl; k < nback; k += G) {
            const Real ux = vx[k], uy = vy[k], uz = vz[k];
            rec_put(a.drec, base + k, qx[k], qy[k], Z3 ? qz[k] : (Real)0, ux, uy, uz, 0u);
            if (do_sample) add_moments(mo, ux, uy, uz);
        }
        if constexpr (MODE == MODE_FUSED) {
            // the move of step s + 1, straight from the pool: particle k of cell c, one per
            // lane at a time, into the bins of half p with its order key
            const MoveCtx<Real> m = move_ctx(a);
            const Origin org = origin_of(m, gc);
            const Half<Real> dst = half_s(a);
            const uint32_t nm = moving && act ? n : 0u;
            const uint32_t nmax = __reduce_max_sync(kFull, nm);
            for (uint32_t k0 = 0; k0 < nmax; k0 += G) {
                const uint32_t k1 = k0 + (uint32_t)gl;
                const bool act1 = k1 < nm;
                Real p1[6] = {0, 0, 0, 0, 0, 0};
                if (act1) {
                    p1[0] = qx[k1]; p1[1] = qy[k1]; if constexpr (Z3) p1[2] = qz[k1];
                    p1[3] = vx[k1]; p1[4] = vy[k1]; p1[5] = vz[k1];
                    if (do_sample) add_moments(mo, p1[3], p1[4], p1[5]);
                }
                uint32_t key1 = 0, ok1 = 0;
                int dir1 = -1;
                if (act1)
                    key1 = move_particle<Real, Z3>(m, org, k1, s + 1u, p1[0], p1[1], p1[2], p1[3], p1[4],
                                                   p1[5], hits, caps, dir1, ok1);
                const bool loc1 = act1 && dir1 < 0;
                const uint32_t arr1 = bin_arrival1(dst.count, key1, loc1, lane);
                if (loc1) {
                    if (arr1 < bin)
                        put_particle<Real, Z3>(dst, (int64_t)key1 * bin + arr1, ok1, p1[0], p1[1], p1[2],
                                               p1[3], p1[4], p1[5]);
                    else
                        lost += 1;
                } else if (act1) {
                    send_particle<Real, Z3>(a.xrec, a.xkey, a.xcount, a.xcap, dir1, key1, ok1, p1[0],
                                            p1[1], p1[2], p1[3], p1[4], p1[5], lost);
                }
            }
            // the arrivals of half p^1 are consumed: their count starts the next step's
            // arrivals (a regenerated cell's count is consumed by LB2DSMC)
            if (moving && act && gl == 0) a.count_d[c] = 0;
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
                // one FP64 addition per sum to the cell's sums copied in at the block's start
                // (each sum has one writer per step)
                cp_async_wait_all();
                __syncwarp(0xFFu << (8 * grp));
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int mq = 3 * gl + q;
                    if (mq < kMoments) a.acc[(size_t)c * kMoments + mq] = s_acc[gi][mq] + widen(t[q]);
                }
            }
        }
        __syncthreads();  // the pool is reused by the next round
    }
    if constexpr (MODE == MODE_FUSED) move_events(a.counters, a.ctrl, hits, caps, lost, lane);
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
        if (nl) atomicAdd(&a.ctrl[CTRL_NACC], nl);
        if (fl) atomicOr(&a.ctrl[CTRL_STATUS], fl);
        // (k_step_end, launched after the pass, publishes the count and advances the step: no
        // block waits here for a grid-wide ticket while it holds its shared memory)
    }
}

template <typename Real, bool BATCH, bool Z3 = false, int MODE = MODE_COLLIDE, int W = kCollideWarps>
__global__ void __launch_bounds__(W * 32, (CollideCfg<Real, W>::MINB))
    k_collide(Launch<DsmcArgs<Real>> L, uint32_t pool) {
    pdl_begin();
    if constexpr (BATCH) {
        const int r = replica_of(L.pre, L.nrep, (int64_t)blockIdx.x);
        collide_block<Real, Z3, MODE, W>(L.tab[r], pool, (int)(blockIdx.x - L.pre[r]));
    } else {
        collide_block<Real, Z3, MODE, W>(L.one, pool, (int)blockIdx.x);
    }
}

// The end of a DSMC step, after its collide pass: the particles the pass counted become the
// live count, and the step and sample counters advance. One thread per context.
template <typename Real, bool BATCH>
__global__ void k_step_end(Launch<DsmcArgs<Real>> L) {
    pdl_begin();
    const int r = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= (BATCH ? L.nrep : 1)) return;
    const DsmcArgs<Real>& a = BATCH ? L.tab[r] : L.one;
    uint32_t* ctrl = a.ctrl;
    const uint32_t s = ctrl[CTRL_STEP];
    ctrl[CTRL_NTOT] = ctrl[CTRL_NACC];
    ctrl[CTRL_NACC] = 0u;
    if (s % (uint32_t)a.sample_every == 0u) ctrl[CTRL_NSAMPLES] += 1u;
    ctrl[CTRL_STEP] = s + 1u;
}

// Appends the particles a streamwise slab received from its neighbours (records and channel
// cells from the slab below, then above) to the bins of their cells in half p^1, after the
// slab's move, with their order keys; then clears the slab's own send counts for its
// next move (the caller has copied its send buffers out by then). A received cell outside the
// slab is skipped and raises HYB_ST_BAD_INPUT.
template <typename Real, bool Z3>
__global__ void __launch_bounds__(256) k_merge(DsmcArgs<Real> a) {
    pdl_begin();
    const unsigned lane = lane_id();
    const uint32_t bin = (uint32_t)a.bin;
    const Half<Real> dst = half_d(a);
    const uint32_t cap = (uint32_t)a.xcap;
    const uint32_t n0 = min(*a.rcount[0], cap), n1 = min(*a.rcount[1], cap);
    const uint32_t total = n0 + n1;
    const uint32_t nz = a.ncz ? (uint32_t)a.ncz : 1u;
    uint32_t lost = 0, bad = 0;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32 * 32;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = w0; i0 < (int64_t)total; i0 += wstride) {  // warp-uniform trip count
        const int64_t i = i0 + lane;
        bool loc = false;
        uint32_t key = 0, tag = 0;
        Real px = 0, py = 0, pz = 0, ux = 0, uy = 0, uz = 0;
        if (i < (int64_t)total) {
            const int d = i < (int64_t)n0 ? 0 : 1;
            const int64_t j = d ? i - n0 : i;
            rec_get(a.rrec[d], j, px, py, pz, ux, uy, uz, tag);
            const uint32_t gk = a.rkey[d][j];
            const uint32_t plane = (uint32_t)a.ncx * (uint32_t)a.ncy_g;
            const uint32_t iz = gk / plane, r = gk - iz * plane;
            const uint32_t iy = r / (uint32_t)a.ncx, ix = r - iy * (uint32_t)a.ncx;
            const int iyl = (int)iy - a.y0;
            if (iyl >= 0 && iyl < a.ncy && iz < nz) {
                key = (iz * (uint32_t)a.ncy + (uint32_t)iyl) * (uint32_t)a.ncx + ix;
                loc = true;
            } else {
                bad += 1;
            }
        }
        const uint32_t arr = bin_arrival1(dst.count, key, loc, lane);
        if (loc) {
            if (arr < bin)
                put_particle<Real, Z3>(dst, (int64_t)key * bin + arr, tag, px, py, pz, ux, uy, uz);
            else
                lost += 1;
        }
    }
    lost = __reduce_add_sync(kFull, lost);
    bad = __reduce_add_sync(kFull, bad);
    if (lane == 0 && (lost | bad))
        atomicOr(&a.ctrl[CTRL_STATUS], (lost ? HYB_ST_CAPACITY : 0u) | (bad ? HYB_ST_BAD_INPUT : 0u));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.xcount[0] = 0u;
        *a.xcount[1] = 0u;
    }
}

// Sets coupled[cells[i]] = v for the listed cells (indices out of range are skipped).
__global__ void k_mark_cells(uint8_t* coupled, const int32_t* cells, int32_t n, int64_t ncells,
                             uint8_t v) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t c = cells[i];
        if (c >= 0 && (int64_t)c < ncells) coupled[c] = v;
    }
}

template <typename Real>
DsmcArgs<Real> make_args(Ctx& c) {
    DsmcArgs<Real> a{};
    const int h = c.cur_p, o = c.cur_p ^ 1;
    a.srec = (Real*)c.st.part[h];
    a.drec = (Real*)c.st.part[o];
    a.count_s = c.st.count[h];
    a.count_d = c.st.count[o];
    a.crmax = (Real*)c.st.crmax;
    a.rem = (Real*)c.st.rem;
    a.nbar_sum = c.st.nbar_sum;
    a.acc = c.st.acc;
    a.ctrl = c.st.ctrl;
    a.counters = c.st.counters;
    a.coupled = c.st.coupled;
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
    a.ncz = c.p.ncz >= 2 ? c.p.ncz : 0;
    a.crmax_init = c.p.crmax_init;
    a.seed = c.p.seed;
    a.y0 = c.p.ncy_global > 0 ? c.p.y0 : 0;
    a.ncy_g = c.p.ncy_global > 0 ? c.p.ncy_global : c.p.ncy;
    a.xcap = (int32_t)c.d.xcap;
    for (int d = 0; d < 2; ++d) {
        char* xs = c.st.xsend[d];
        char* xr = c.st.xrecv[d];
        const size_t keys = 256 + (size_t)c.d.xcap * kRec * sizeof(Real);
        a.xcount[d] = c.d.xcap ? (uint32_t*)xs : nullptr;
        a.xrec[d] = c.d.xcap ? (Real*)(xs + 256) : nullptr;
        a.xkey[d] = c.d.xcap ? (uint32_t*)(xs + keys) : nullptr;
        a.rcount[d] = c.d.xcap ? (const uint32_t*)xr : nullptr;
        a.rrec[d] = c.d.xcap ? (const Real*)(xr + 256) : nullptr;
        a.rkey[d] = c.d.xcap ? (const uint32_t*)(xr + keys) : nullptr;
    }
    return a;
}

int grid_for(const Ctx& c, int64_t work, int threads, int per_sm) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)c.num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// Shared memory of a collide block: the pool (pool_reals Real and one u32 per slot) and one
// pass of NTC candidates (u32 and 4 Real each).
template <typename Real, bool Z3, int W = kCollideWarps>
size_t collide_smem(uint32_t pool, uint32_t bin) {
    constexpr int NC = W * (32 / kGroup);
    const size_t cand = (size_t)NC * kChainSteps * (4 + 4 * sizeof(Real));
    const size_t bits = ((size_t)NC * (bitmap_words<Z3>(bin) * 5 + (kFarList + 1) * 4) + 15) / 16 * 16;
    return (size_t)pool * (pool_reals<Z3>() * sizeof(Real)) + (cand > bits ? cand : bits);
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
    if (c.st.coupled) cudaMemsetAsync(c.st.coupled, 0, (size_t)c.d.ncells, c.stream);
    for (int d = 0; d < 2 && c.d.xcap; ++d) {  // the exchange counts start at zero
        cudaMemsetAsync(c.st.xsend[d], 0, 4, c.stream);
        cudaMemsetAsync(c.st.xrecv[d], 0, 4, c.stream);
    }
    return cudaGetLastError();
}

template <typename Real, bool Z3>
cudaError_t move_impl(Ctx& c, int p) {
    const int save = c.cur_p;
    c.cur_p = p;
    Launch<DsmcArgs<Real>> L{};
    L.one = make_args<Real>(c);
    c.cur_p = save;
    L.total = c.d.ncells;
    prof_begin(c, K_MOVE);
    // one source cell per warp (the hardware schedules the blocks as resources free up)
    const cudaError_t e = launch_pdl(k_move<Real, false, Z3>, dim3(grid_for(c, c.d.ncells * 32, 256, 64)),
                                     dim3(256), 0, c.stream, L);
    prof_end(c, K_MOVE);
    return e;
}

template <typename Real, bool Z3, int MODE, int W>
cudaError_t collide_impl_w(Ctx& c, int p) {
    const int save = c.cur_p;
    c.cur_p = p;
    Launch<DsmcArgs<Real>> L{};
    L.one = make_args<Real>(c);
    c.cur_p = save;
    constexpr int NC = W * (32 / kGroup);
    const uint32_t pool = collide_pool(c, W);
    const size_t smem = collide_smem<Real, Z3, W>(pool, (uint32_t)c.d.bin);
    // (dynamic and static shared memory together may exceed the default 48 KB)
    cudaError_t e = cudaFuncSetAttribute(k_collide<Real, false, Z3, MODE, W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((c.d.ncells + NC - 1) / NC);
    L.total = grid;
    constexpr int kid = MODE == MODE_FUSED ? K_FUSED : K_COLLIDE;
    prof_begin(c, kid);
    e = launch_pdl(k_collide<Real, false, Z3, MODE, W>, dim3(grid), dim3(W * 32), smem, c.stream, L, pool);
    prof_end(c, kid);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_step_end<Real, false>, dim3(1), dim3(32), 0, c.stream, L);
}

// The context's collide block shape: 8 warps (32 cells) or 4 (16 cells).
template <typename Real, bool Z3, int MODE>
cudaError_t collide_impl(Ctx& c, int p) {
    return c.collide_warps == 4 ? collide_impl_w<Real, Z3, MODE, 4>(c, p) : collide_impl_w<Real, Z3, MODE, 8>(c, p);
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

cudaError_t launch_dsmc_move(Ctx& c, int p) {
    if (c.p.ncz >= 2) return c.p.real_bytes == 4 ? move_impl<float, true>(c, p) : move_impl<double, true>(c, p);
    return c.p.real_bytes == 4 ? move_impl<float, false>(c, p) : move_impl<double, false>(c, p);
}

cudaError_t launch_dsmc_collide(Ctx& c, int p) {
    if (c.p.ncz >= 2)
        return c.p.real_bytes == 4 ? collide_impl<float, true, MODE_COLLIDE>(c, p)
                                   : collide_impl<double, true, MODE_COLLIDE>(c, p);
    return c.p.real_bytes == 4 ? collide_impl<float, false, MODE_COLLIDE>(c, p)
                               : collide_impl<double, false, MODE_COLLIDE>(c, p);
}

cudaError_t launch_dsmc_fused(Ctx& c, int p) {
    if (c.p.ncz >= 2)
        return c.p.real_bytes == 4 ? collide_impl<float, true, MODE_FUSED>(c, p)
                                   : collide_impl<double, true, MODE_FUSED>(c, p);
    return c.p.real_bytes == 4 ? collide_impl<float, false, MODE_FUSED>(c, p)
                               : collide_impl<double, false, MODE_FUSED>(c, p);
}

cudaError_t launch_dsmc_step(Ctx& c) {
    cudaError_t e = launch_dsmc_move(c, c.cur_p);
    if (e != cudaSuccess) return e;
    return launch_dsmc_collide(c, c.cur_p);
}

namespace {
template <typename Real, bool Z3>
cudaError_t merge_impl(Ctx& c, int p) {
    const int save = c.cur_p;
    c.cur_p = p;
    const DsmcArgs<Real> a = make_args<Real>(c);
    c.cur_p = save;
    return launch_pdl(k_merge<Real, Z3>, dim3(grid_for(c, c.d.xcap * 2, 256, 4)), dim3(256), 0,
                      c.stream, a);
}
}  // namespace

cudaError_t launch_dsmc_merge(Ctx& c, int p) {
    if (!c.d.xcap) return cudaSuccess;
    if (c.p.ncz >= 2) return c.p.real_bytes == 4 ? merge_impl<float, true>(c, p) : merge_impl<double, true>(c, p);
    return c.p.real_bytes == 4 ? merge_impl<float, false>(c, p) : merge_impl<double, false>(c, p);
}

cudaError_t launch_mark_cells(Ctx& c, const int32_t* cells, int32_t n, uint8_t v) {
    if (n <= 0) return cudaSuccess;
    k_mark_cells<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(c.st.coupled, cells, n,
                                                                    c.d.ncells, v);
    return cudaGetLastError();
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

namespace {
// Blocks of a collide kernel resident per SM at `smem` bytes of dynamic shared memory (the
// kernel's limit is raised to it first, as for a launch); 0 if the query fails.
template <typename Kern>
int collide_per_sm(Kern kernel, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
        return 0;
    return per_sm;
}
}  // namespace

// Whether the fused pass's grid fills the GPU: at least as many blocks of 32 cells as fit on
// it at once. Below that a launch is one partial wave whose time is the latency of its
// slowest block, which the fused pass lengthens (a collide and a move in one block), and two
// separate passes are faster.
namespace {
template <int W>
bool fused_fills_gpu_w(const Ctx& c) {
    constexpr int NC = W * (32 / kGroup);
    const uint32_t pool = collide_pool(c, W);
    const uint32_t bin = (uint32_t)c.d.bin;
    const bool z3 = c.p.ncz >= 2;
    int per_sm;
    if (c.p.real_bytes == 4)
        per_sm = z3 ? collide_per_sm(k_collide<float, false, true, MODE_FUSED, W>, W * 32,
                                     collide_smem<float, true, W>(pool, bin))
                    : collide_per_sm(k_collide<float, false, false, MODE_FUSED, W>, W * 32,
                                     collide_smem<float, false, W>(pool, bin));
    else
        per_sm = z3 ? collide_per_sm(k_collide<double, false, true, MODE_FUSED, W>, W * 32,
                                     collide_smem<double, true, W>(pool, bin))
                    : collide_per_sm(k_collide<double, false, false, MODE_FUSED, W>, W * 32,
                                     collide_smem<double, false, W>(pool, bin));
    if (per_sm < 1) return true;
    const int64_t blocks = (c.d.ncells + NC - 1) / NC;
    return blocks >= (int64_t)per_sm * c.num_sms;
}
}  // namespace

bool dsmc_fused_fills_gpu(const Ctx& c) {
    return c.collide_warps == 4 ? fused_fills_gpu_w<4>(c) : fused_fills_gpu_w<8>(c);
}

// Pool slots of a collide block of `warps` warps (4 cells each): room for 1.1 ppc per cell on
// average (the cells' counts add up to about NC ppc with a spread of sqrt(NC ppc); a block
// whose cells do not fit takes the pool one cell at a time), and at least one full bin.
uint32_t collide_pool(const Ctx& c, int warps) {
    const int NC = warps * (32 / kGroup);
    uint32_t pool = (uint32_t)(((int64_t)NC * c.p.ppc * 11 / 10 + 31) / 32 * 32);
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
    Launch<DsmcArgs<Real>> L{};
    L.tab = (const DsmcArgs<Real>*)b.dsmc[cur_p];
    L.nrep = b.nrep;
    cudaError_t e;
    if (b.collide_block == 128) {  // blocks of 16 cells
        L.pre = b.pre_blocks4;
        L.total = b.tot_blocks4;
        const size_t smem = collide_smem<Real, false, 4>(b.pool4, b.maxbin);
        auto k = k_collide<Real, true, false, MODE_COLLIDE, 4>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = launch_pdl(k, dim3((unsigned)L.total), dim3(128), smem, b.stream, L, b.pool4);
    } else {  // blocks of 32 cells
        L.pre = b.pre_blocks;
        L.total = b.tot_blocks;
        const size_t smem = collide_smem<Real, false, 8>(b.pool, b.maxbin);
        auto k = k_collide<Real, true, false, MODE_COLLIDE, 8>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = launch_pdl(k, dim3((unsigned)L.total), dim3(256), smem, b.stream, L, b.pool);
    }
    if (e != cudaSuccess) return e;
    return launch_pdl(k_step_end<Real, true>, dim3((unsigned)((L.nrep + 127) / 128)), dim3(128), 0,
                      b.stream, L);
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
