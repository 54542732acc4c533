// DSMC kernels: initialisation, move with diffuse isothermal walls, stable counting sort by
// cell, no-time-counter hard-sphere collisions and per-cell Hermite-moment sampling.
//
// One DSMC step (Sec. 5, the NTC scheme of Bird that the paper uses) is five launches:
//   k_move        per particle: body-force kick, free flight, diffuse wall re-emission
//                 (Sec. 3.1), periodic wrap; new cell key; warp-aggregated arrival count.
//   k_tile_sums   per 4096-cell tile: sum of the per-cell counts.
//   k_scan        per tile: exclusive scan -> cell_start; counts cleared for the next step.
//   k_rank        per particle: perm[cell_start[key] + arrival] = slot.
//   k_collide     one warp per cell: the cell's slots are put back in ascending old-slot
//                 order (so the sort is stable whatever order the atomics gave), gathered
//                 into the other half of the ping-pong buffer, collided by NTC
//                 (Eq. collisionnumber) in shared memory, written out, and their moment
//                 sums 1, v, vv, vvv added to the FP64 cumulative sums (Sec. 2.1, Fig. 1).
// This file is compiled without FMA contraction so that positions, cell keys, pair choices
// and post-collision velocities are the IEEE float (or double) results of the written
// expressions.
#include "hyb_internal.cuh"

namespace hyb {

namespace {

template <typename Real>
__device__ __forceinline__ void reemit(uint64_t seed, uint32_t slot, uint32_t s, int bounce, Real sign,
                                       Real& ux, Real& uy, Real& uz) {
    const uint4 r = draw(seed, slot, s, TAG_WALL, (uint32_t)bounce, 0);
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

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t* sh) {
    v = __reduce_add_sync(kFull, v);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane_id() == 0) sh[w] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int i = 0; i < nw; ++i) t += sh[i];
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------------------------------
template <typename Real>
__global__ void k_init_particles(DsmcArgs<Real> a) {
    const int64_t n = (int64_t)a.ncells * a.ppc;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(s / a.ppc), k = (uint32_t)(s % a.ppc);
        const int ix = (int)(c % (uint32_t)a.ncx), iy = (int)(c / (uint32_t)a.ncx);
        const uint4 rp = draw(a.seed, c, 0, TAG_INIT_POS, k, 0);
        a.dx[s] = (Real)ix + (Real)u01f(rp.x);
        a.dy[s] = (Real)iy + (Real)u01f(rp.y);
        const uint4 rv = draw(a.seed, c, 0, TAG_INIT_VEL, k, 0);
        Real n0, n1, n2, n3;
        gauss_pair<Real>(rv.x, rv.y, n0, n1);
        gauss_pair<Real>(rv.z, rv.w, n2, n3);
        a.dvx[s] = n0;
        a.dvy[s] = n1;
        a.dvz[s] = n2;
    }
}

template <typename Real>
__global__ void k_init_cells(DsmcArgs<Real> a) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= a.ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        a.cell_start[c] = (uint32_t)(c * a.ppc);
        if (c < a.ncells) {
            a.count[c] = 0;
            a.crmax[c] = (Real)a.crmax_init;
            a.rem[c] = (Real)0;
            a.nbar_sum[c] = 0u;
            for (int m = 0; m < kMoments; ++m) a.acc[c * kMoments + m] = 0.0;
        }
        if (c == 0) {
            for (int w = 0; w < CTRL_WORDS; ++w) a.ctrl[w] = 0;
            a.ctrl[CTRL_NTOT] = (uint32_t)((int64_t)a.ncells * a.ppc);
            for (int w = 0; w < HYB_NCOUNTERS; ++w) a.counters[w] = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Move (kick, drift, walls, wrap), cell key, arrival index.
template <typename Real>
__global__ void __launch_bounds__(256) k_move(DsmcArgs<Real> a) {
    const uint32_t n = a.ctrl[CTRL_NTOT];
    const uint32_t s = a.ctrl[CTRL_STEP];
    const Real H = (Real)a.ncx, L = (Real)a.ncy;
    const Real g = (Real)a.g_step, dt = (Real)a.dt;
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    uint32_t hits = 0, caps = 0;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        uint32_t k = kDeadKey;
        if (i < n) {
            Real px = a.mx[i];
            if (px >= (Real)0) {
                Real py = a.my[i];
                Real ux = a.mvx[i], uy = a.mvy[i] + g, uz = a.mvz[i];
                Real t = dt;
                for (int b = 0;; ++b) {
                    const Real xn = px + ux * t;
                    const bool left = xn < (Real)0;
                    const bool right = xn > H;
                    if (!left && !right) {
                        px = xn;
                        py = py + uy * t;
                        break;
                    }
                    if (b == kMaxBounces) {
                        caps += 1;
                        px = left ? (Real)0 : H;
                        py = py + uy * t;
                        break;
                    }
                    hits += 1;
                    const Real th = left ? px / (-ux) : (H - px) / ux;
                    py = py + uy * th;
                    px = left ? (Real)0 : H;
                    t = t - th;
                    if (t < (Real)0) t = (Real)0;
                    reemit(a.seed, i, s, b, left ? (Real)1 : (Real)-1, ux, uy, uz);
                }
                if (py < (Real)0 || py >= L) {
                    py = py - L * floor(py / L);
                    if (py < (Real)0) py = py + L;
                    if (py >= L) py = py - L;
                }
                a.mx[i] = px;
                a.my[i] = py;
                a.mvx[i] = ux;
                a.mvy[i] = uy;
                a.mvz[i] = uz;
                int ix = (int)floor(px), iy = (int)floor(py);
                ix = ix < 0 ? 0 : (ix > a.ncx - 1 ? a.ncx - 1 : ix);
                iy = iy < 0 ? 0 : (iy > a.ncy - 1 ? a.ncy - 1 : iy);
                k = (uint32_t)(iy * a.ncx + ix);
            }
            a.key[i] = k;
        }
        const bool live = k != kDeadKey;
        const unsigned m = __ballot_sync(kFull, live);
        if (live) {
            // lanes with the same cell share one atomic; arrival = base + rank among them
            const unsigned peers = __match_any_sync(m, k);
            const int leader = __ffs(peers) - 1;
            uint32_t b0 = 0;
            if ((int)lane == leader) b0 = atomicAdd(&a.count[k], (uint32_t)__popc(peers));
            b0 = __shfl_sync(peers, b0, leader);
            a.arrival[i] = b0 + (uint32_t)__popc(peers & lt);
        }
    }
    hits = __reduce_add_sync(kFull, hits);
    caps = __reduce_add_sync(kFull, caps);
    if (lane == 0) {
        if (hits) atomicAdd(&a.counters[HYB_C_WALL_HITS], (unsigned long long)hits);
        if (caps) {
            atomicAdd(&a.counters[HYB_C_BOUNCE_CAP], (unsigned long long)caps);
            atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BOUNCE_CAP);
        }
    }
}

__global__ void __launch_bounds__(256) k_tile_sums(const uint32_t* count, uint32_t* tile_sum,
                                                   int ncells) {
    __shared__ uint32_t sh[8];
    const int c0 = blockIdx.x * kScanTile;
    const int c1 = min(c0 + kScanTile, ncells);
    uint32_t s = 0;
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) s += count[c];
    s = block_sum_u32(s, sh);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = s;
}

// Exclusive scan of one tile of counts, offset by the sum of the lower tiles.
template <typename Real>
__global__ void __launch_bounds__(256) k_scan(DsmcArgs<Real> a) {
    constexpr int PER = kScanTile / 256;
    __shared__ uint32_t sh[8];
    __shared__ uint32_t warp_tot[8];
    const int t = blockIdx.x;
    uint32_t pre = 0;
    for (int u = threadIdx.x; u < t; u += blockDim.x) pre += a.tile_sum[u];
    pre = block_sum_u32(pre, sh);
    const int c0 = t * kScanTile + threadIdx.x * PER;
    uint32_t v[PER];
    uint32_t loc = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int c = c0 + k;
        v[k] = c < a.ncells ? a.count[c] : 0u;
        loc += v[k];
    }
    // block exclusive scan of loc
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    uint32_t incl = loc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, off);
        if ((int)lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    uint32_t wpre = 0;
    for (int i = 0; i < w; ++i) wpre += warp_tot[i];
    uint32_t run = pre + wpre + incl - loc;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int c = c0 + k;
        if (c < a.ncells) {
            a.cell_start[c] = run;
            a.count[c] = 0;
        }
        run += v[k];
    }
    if (t == a.ntiles - 1 && threadIdx.x == blockDim.x - 1) a.cell_start[a.ncells] = run;
    if (t == 0 && threadIdx.x == 0) {
        const uint32_t s = a.ctrl[CTRL_STEP];
        if (s % (uint32_t)a.sample_every == 0) a.ctrl[CTRL_NSAMPLES] += 1;
        a.ctrl[CTRL_STEP] = s + 1;
    }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_rank(DsmcArgs<Real> a) {
    const uint32_t n = a.ctrl[CTRL_NTOT];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = a.key[i];
        if (k != kDeadKey) a.perm[a.cell_start[k] + a.arrival[i]] = i;
    }
}

// ---------------------------------------------------------------------------------------
// One warp per cell: stable order, gather, NTC collisions, write-out, moment sums.
constexpr int kCollideWarps = 4;

// Ascending bitonic sort of 32 R keys held R per lane (key r of a lane at position
// lane + 32 r). All loops have constant trip counts and unroll, so the keys stay in registers.
template <int R>
__device__ __forceinline__ void bitonic_sort(uint32_t (&v)[R]) {
    constexpr int N = 32 * R;
    const int lane = (int)lane_id();
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j >> 5;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int o = r ^ jr;
                    if (r < o) {
                        const bool asc = ((lane + 32 * r) & k) == 0;
                        const uint32_t lo = min(v[r], v[o]), hi = max(v[r], v[o]);
                        v[r] = asc ? lo : hi;
                        v[o] = asc ? hi : lo;
                    }
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t o = __shfl_xor_sync(kFull, v[r], j);
                    const bool asc = ((lane + 32 * r) & k) == 0;
                    v[r] = (lower == asc) ? min(v[r], o) : max(v[r], o);
                }
            }
        }
    }
}

// Sort the cell's n <= 32 R slots from perm and gather them into the destination half.
template <typename Real, int R>
__device__ __forceinline__ void sort_gather(const DsmcArgs<Real>& a, uint32_t start, uint32_t n,
                                            Real* vx, Real* vy, Real* vz) {
    const unsigned lane = lane_id();
    uint32_t v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t k = lane + 32u * r;
        v[r] = k < n ? a.perm[start + k] : 0xFFFFFFFFu;
    }
    bitonic_sort<R>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t k = lane + 32u * r;
        if (k < n) {
            const uint32_t src = v[r];
            a.dx[start + k] = a.sx[src];
            a.dy[start + k] = a.sy[src];
            vx[k] = a.svx[src];
            vy[k] = a.svy[src];
            vz[k] = a.svz[src];
        }
    }
}

template <typename Real, int MAXP>
__global__ void __launch_bounds__(kCollideWarps * 32) k_collide(DsmcArgs<Real> a) {
    __shared__ uint32_t s_in[kCollideWarps][MAXP];
    __shared__ Real s_v[kCollideWarps][3][MAXP];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const uint32_t s = a.ctrl[CTRL_STEP] - 1u;
    const bool do_sample = (s % (uint32_t)a.sample_every) == 0u;
    const Real coll_dt = (Real)a.coll_dt;
    unsigned long long ncand_tot = 0, ncoll_tot = 0;
    uint32_t flags = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl[CTRL_NTOT] = a.cell_start[a.ncells];

    for (int c = blockIdx.x * kCollideWarps + w; c < a.ncells; c += gridDim.x * kCollideWarps) {
        const uint32_t start = a.cell_start[c];
        const uint32_t n = a.cell_start[c + 1] - start;
        const bool small = n <= (uint32_t)MAXP;
        Real* vx = small ? s_v[w][0] : a.dvx + start;
        Real* vy = small ? s_v[w][1] : a.dvy + start;
        Real* vz = small ? s_v[w][2] : a.dvz + start;
        // 1. the cell's old slots in ascending order, 2. gathered into the other half
        if (n <= 32) {
            sort_gather<Real, 1>(a, start, n, vx, vy, vz);
        } else if (n <= 64) {
            sort_gather<Real, 2>(a, start, n, vx, vy, vz);
        } else if (n <= 128) {
            sort_gather<Real, 4>(a, start, n, vx, vy, vz);
        } else {
            // rank of each slot = number of smaller slots in the cell
            uint32_t* srt = a.arrival + start;
            const uint32_t* in = small ? s_in[w] : a.perm + start;
            if (small)
                for (uint32_t k = lane; k < n; k += 32) s_in[w][k] = a.perm[start + k];
            __syncwarp();
            for (uint32_t k = lane; k < n; k += 32) {
                const uint32_t v = in[k];
                uint32_t r = 0;
                for (uint32_t m = 0; m < n; ++m) r += in[m] < v ? 1u : 0u;
                srt[r] = v;
            }
            __syncwarp();
            for (uint32_t k = lane; k < n; k += 32) {
                const uint32_t src = srt[k];
                a.dx[start + k] = a.sx[src];
                a.dy[start + k] = a.sy[src];
                vx[k] = a.svx[src];
                vy[k] = a.svy[src];
                vz[k] = a.svz[src];
            }
        }
        __syncwarp();
        // 3. NTC: N_cand = 1/2 N Nbar F_N (sigma c_r)_max dt / V_c + remainder
        uint32_t nsel = 0;
        Real cm = (Real)0;
        if (lane == 0) {
            const uint32_t nb = a.nbar_sum[c] + n;
            a.nbar_sum[c] = nb;
            cm = a.crmax[c];
            if (n > 32767u) {
                flags |= HYB_ST_CELL_OVERFLOW;  // pair indices are packed in 15 and 16 bits
            } else if (n >= 2) {
                const Real nbar = (Real)nb / (Real)(s + 1u);
                const Real ncand = (Real)0.5 * (Real)n * nbar * cm * coll_dt + a.rem[c];
                const Real fl = floor(ncand);
                a.rem[c] = ncand - fl;
                if (fl > (Real)16777215) {
                    nsel = 16777215u;
                    flags |= HYB_ST_CELL_OVERFLOW;
                } else {
                    nsel = (uint32_t)fl;
                }
            }
        }
        nsel = __shfl_sync(kFull, nsel, 0);
        cm = __shfl_sync(kFull, cm, 0);
        uint32_t ncoll = 0;
        for (uint32_t ch = 0; ch < nsel; ch += 32) {
            // lanes draw 32 candidates in parallel; they are applied in order below
            const uint32_t k = ch + lane;
            uint32_t ij = 0;
            Real R = (Real)0, nx = (Real)0, ny = (Real)0, nz = (Real)0;
            if (k < nsel) {
                const uint4 r = draw(a.seed, (uint32_t)c, s, TAG_NTC_PAIR, k, 0);
                const uint32_t ci = uindex(r.x, n);
                uint32_t cj = uindex(r.y, n - 1u);
                if (cj >= ci) cj += 1u;
                R = (Real)u01f(r.z);
                const int ok = unit_vector(a.seed, (uint32_t)c, s, k, nx, ny, nz);
                ij = ci | (cj << 15) | (ok ? 0u : 0x80000000u);
            }
            const uint32_t cnt = min(32u, nsel - ch);
            for (uint32_t m = 0; m < cnt; ++m) {
                const uint32_t ijm = __shfl_sync(kFull, ij, m);
                const uint32_t i = ijm & 0x7FFFu, j = (ijm >> 15) & 0xFFFFu;
                const Real Rm = __shfl_sync(kFull, R, m);
                const Real ax = vx[i], ay = vy[i], az = vz[i];
                const Real bx = vx[j], by = vy[j], bz = vz[j];
                const Real ddx = ax - bx, ddy = ay - by, ddz = az - bz;
                const Real cr = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                if (cr > cm) cm = cr;
                const bool acc_pair = cr > Rm * cm;
                if (acc_pair) {
                    const Real nxm = __shfl_sync(kFull, nx, m);
                    const Real nym = __shfl_sync(kFull, ny, m);
                    const Real nzm = __shfl_sync(kFull, nz, m);
                    if (ijm & 0x80000000u) {
                        flags |= HYB_ST_SCATTER_CAP;
                    } else {
                        __syncwarp();
                        if (lane == 0) {
                            const Real cx = (ax + bx) * (Real)0.5;
                            const Real cy = (ay + by) * (Real)0.5;
                            const Real cz = (az + bz) * (Real)0.5;
                            const Real h = cr * (Real)0.5;
                            vx[i] = cx + h * nxm;
                            vy[i] = cy + h * nym;
                            vz[i] = cz + h * nzm;
                            vx[j] = cx - h * nxm;
                            vy[j] = cy - h * nym;
                            vz[j] = cz - h * nzm;
                        }
                        __syncwarp();
                        ncoll += 1;
                    }
                }
            }
        }
        if (lane == 0) {
            a.crmax[c] = cm;
            ncand_tot += nsel;
            ncoll_tot += ncoll;
        }
        // 4. write-out and moment sums
        Real mo[kMoments];
#pragma unroll
        for (int q = 0; q < kMoments; ++q) mo[q] = (Real)0;
        for (uint32_t k = lane; k < n; k += 32) {
            const Real ux = vx[k], uy = vy[k], uz = vz[k];
            if (small) {
                a.dvx[start + k] = ux;
                a.dvy[start + k] = uy;
                a.dvz[start + k] = uz;
            }
            if (do_sample) {
                const Real xx = ux * ux, yy = uy * uy, zz = uz * uz;
                const Real xy = ux * uy, xz = ux * uz, yz = uy * uz;
                mo[0] += (Real)1;
                mo[1] += ux; mo[2] += uy; mo[3] += uz;
                mo[4] += xx; mo[5] += xy; mo[6] += xz; mo[7] += yy; mo[8] += yz; mo[9] += zz;
                mo[10] += xx * ux; mo[11] += xx * uy; mo[12] += xx * uz; mo[13] += yy * ux;
                mo[14] += xy * uz; mo[15] += zz * ux; mo[16] += yy * uy; mo[17] += yy * uz;
                mo[18] += zz * uy; mo[19] += zz * uz;
            }
        }
        if (do_sample) {
            Real mine = (Real)0;
#pragma unroll
            for (int q = 0; q < kMoments; ++q) {
                Real v = mo[q];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
                if ((int)lane == q) mine = v;
            }
            if (lane < (unsigned)kMoments) a.acc[(size_t)c * kMoments + lane] += (double)mine;
        }
        __syncwarp();
    }
    // event counters
    if (lane == 0) {
        if (ncand_tot) atomicAdd(&a.counters[HYB_C_CANDIDATES], ncand_tot);
        if (ncoll_tot) atomicAdd(&a.counters[HYB_C_COLLISIONS], ncoll_tot);
    }
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0 && flags) atomicOr(&a.ctrl[CTRL_STATUS], flags);
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
    a.mx = (Real*)c.st.px[h];
    a.my = (Real*)c.st.py[h];
    a.mvx = (Real*)c.st.pvx[h];
    a.mvy = (Real*)c.st.pvy[h];
    a.mvz = (Real*)c.st.pvz[h];
    a.dx = (Real*)c.st.px[o];
    a.dy = (Real*)c.st.py[o];
    a.dvx = (Real*)c.st.pvx[o];
    a.dvy = (Real*)c.st.pvy[o];
    a.dvz = (Real*)c.st.pvz[o];
    a.key = c.st.key;
    a.arrival = c.st.arrival;
    a.perm = c.st.perm;
    a.count = c.st.count;
    a.cell_start = c.st.cell_start;
    a.tile_sum = c.st.tile_sum;
    a.crmax = (Real*)c.st.crmax;
    a.rem = (Real*)c.st.rem;
    a.nbar_sum = c.st.nbar_sum;
    a.acc = c.st.acc;
    a.ctrl = c.st.ctrl;
    a.counters = c.st.counters;
    a.ncx = c.p.ncx;
    a.ncy = c.p.ncy;
    a.ncells = (int32_t)c.d.ncells;
    a.ntiles = (int32_t)c.L.ntiles;
    a.sample_every = c.p.sample_every;
    a.ppc = c.p.ppc;
    a.capacity = c.d.capacity;
    a.dt = c.d.dt;
    a.g_step = c.d.g_step;
    a.coll_dt = c.d.coll_dt;
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
    // initial particles go to half 0
    c.cur_p = 1;
    DsmcArgs<Real> a = make_args<Real>(c);
    c.cur_p = 0;
    const int64_t n = c.d.ncells * c.p.ppc;
    k_init_particles<Real><<<grid_for(c, n, 256, 16), 256, 0, c.stream>>>(a);
    k_init_cells<Real><<<grid_for(c, c.d.ncells + 1, 256, 16), 256, 0, c.stream>>>(a);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t step_impl(Ctx& c) {
    DsmcArgs<Real> a = make_args<Real>(c);
    const int64_t cap = c.d.capacity;
    prof_begin(c, K_MOVE);
    k_move<Real><<<grid_for(c, cap, 256, 8), 256, 0, c.stream>>>(a);
    prof_end(c, K_MOVE);
    prof_begin(c, K_TILE_SUMS);
    k_tile_sums<<<(int)c.L.ntiles, 256, 0, c.stream>>>(a.count, a.tile_sum, a.ncells);
    prof_end(c, K_TILE_SUMS);
    prof_begin(c, K_SCAN);
    k_scan<Real><<<(int)c.L.ntiles, 256, 0, c.stream>>>(a);
    prof_end(c, K_SCAN);
    prof_begin(c, K_RANK);
    k_rank<Real><<<grid_for(c, cap, 256, 8), 256, 0, c.stream>>>(a);
    prof_end(c, K_RANK);
    constexpr int MAXP = sizeof(Real) == 4 ? 256 : 128;
    prof_begin(c, K_COLLIDE);
    k_collide<Real, MAXP>
        <<<grid_for(c, c.d.ncells * 32, kCollideWarps * 32, 16), kCollideWarps * 32, 0, c.stream>>>(a);
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
    return (c.p.real_bytes == 4) ? step_impl<float>(c) : step_impl<double>(c);
}

cudaError_t launch_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n,
                                cudaStream_t s) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_debug_philox<<<(int)g, 256, 0, s>>>(ctr, seed, out, n);
    return cudaGetLastError();
}

}  // namespace hyb
