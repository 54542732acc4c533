// The two kinetic mappings of Sec. 2. The Grad/Hermite coefficients are solved in FP64;
// populations and particle state are Real (float or double).
//
// k_d2l (DSMC2LB, Sec. 2.1): one thread per coupling node. The cumulative sums of the
// node's DSMC cell give rho = <N>/ppc, the per-particle raw moments <v>, <vv>, <vvv>, and
// the raw Hermite coefficients a0 = rho, a1 = rho <v>, a2 = rho(<vv> - I),
// a3 = rho(<vvv> - sym(<v> I)) (FP64); the populations f_a = w_a sum_{n<=N} a^(n):H^(n)(xi_a)/n!
// (Eq. discretefunctions) are evaluated in the state precision.
//
// LB2DSMC (Sec. 2.2, Table 1) in two launches:
//   k_l2d_coef   one warp per coupling cell: mean populations of the cell's lb_ratio^2
//                nodes, rho and u, the comoving coefficients a2 = sum f c c / rho - I and
//                a3 = sum f c c c / rho (c = xi - u), M, C = 1 + 30 M (Eq. C), and the
//                particle count floor(rho ppc + U) (FP64, lanes over populations);
//   k_l2d_sample one warp per coupling cell: the cell's trial stream is evaluated 32 trials
//                at a time: Box-Muller xi from the unit Maxwellian, accepted when
//                C R <= G(xi), G = 1 + a2:H2/2 + a3:H3/6 (Eq. distr_outeq) in the state
//                precision; the k-th accepted trial becomes the k-th particle of the cell's
//                bin (replacing the old ones), velocity xi + u (Eq. step6 in c_th units),
//                position uniform in the cell from the same trial's draws.
// Draws are keyed by (cell, step, purpose, trial index), so the results do not depend on
// the launch shape.
#include "hyb_internal.cuh"

// Fixed scratch of map_lbm_to_dsmc_noalloc: one Grad record per coupling cell, for callers
// that cannot hand the library any device memory beyond the state itself. The array lives
// in every device that loads the library until the process exits. Host code must not pass
// `g_l2d_scratch` itself to a kernel (on the host it names a stand-in, not device memory):
// its device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) hyb::GradRec g_l2d_scratch[HYB_NOALLOC_MAX_CELLS];

namespace hyb {

namespace {

template <class LAT>
__host__ __device__ constexpr int E(int a, int i) {
    return LatTab<LAT>::e(a, i);
}

// Lattice table in shared memory, for lanes that each handle a different population.
template <class LAT>
__device__ __forceinline__ void load_lattice(int* se, double* sw) {
    for (int q = threadIdx.x; q < LAT::Q; q += blockDim.x) {
        se[3 * q] = LatTab<LAT>::e(q, 0);
        se[3 * q + 1] = LatTab<LAT>::e(q, 1);
        se[3 * q + 2] = LatTab<LAT>::e(q, 2);
        sw[q] = LatTab<LAT>::w(q);
    }
}

// DSMC2LB: one warp per coupling node. Lanes 0-19 read the cell's 20 sums; the FP64
// coefficient solve is spread over the lanes (one coefficient each); the 19 coefficients
// are broadcast and each lane evaluates one or two populations in the state precision.
template <typename Real, class LAT>
__global__ void __launch_bounds__(128) k_d2l(MapArgs<Real> a) {
    __shared__ int se[3 * LAT::Q];
    __shared__ double sw[LAT::Q];
    load_lattice<LAT>(se, sw);
    __syncthreads();
    const unsigned lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t S = a.ctrl[CTRL_NSAMPLES];
    constexpr double R = lat_r<LAT>();
    for (int t = gw; t < a.n; t += nw) {
        const int32_t node = a.list[t];
        if (node < 0 || (int64_t)node >= a.nnodes) {
            if (lane == 0) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            continue;
        }
        const int x = node % a.nx, y = node / a.nx;
        const int64_t cell = (int64_t)(y / a.lb_ratio) * a.ncx + (x / a.lb_ratio);
        const double* m = a.acc + cell * kMoments;
        const double mk = lane < (unsigned)kMoments ? m[lane] : 0.0;
        const double NS = __shfl_sync(kFull, mk, 0);
        if (S == 0 || !(NS > 0.0)) {
            if (lane == 0) atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            continue;
        }
        // FP64 coefficient solve, one coefficient per lane:
        // lane 0: rho; 1-3: a1 = rho <v>; 4-9: a2 = rho(<vv> - I); 10-19: a3 = rho(<vvv> - sym(<v> I))
        const double rho = (NS / (double)S) / (double)a.ppc;
        const double iNS = 1.0 / NS;
        const double m1x = __shfl_sync(kFull, mk, 1) * iNS;
        const double m1y = __shfl_sync(kFull, mk, 2) * iNS;
        const double m1z = __shfl_sync(kFull, mk, 3) * iNS;
        double sub = 0.0;
        switch (lane) {
            case 4: case 7: case 9: sub = 1.0; break;        // xx yy zz
            case 10: sub = 3 * m1x; break;                   // xxx
            case 11: sub = m1y; break;                       // xxy
            case 12: sub = m1z; break;                       // xxz
            case 13: sub = m1x; break;                       // xyy
            case 15: sub = m1x; break;                       // xzz
            case 16: sub = 3 * m1y; break;                   // yyy
            case 17: sub = m1z; break;                       // yyz
            case 18: sub = m1y; break;                       // yzz
            case 19: sub = 3 * m1z; break;                   // zzz
            default: break;
        }
        const Real coef = lane == 0 ? (Real)rho : (Real)(rho * (mk * iNS - sub));
        Real cf[kMoments];
#pragma unroll
        for (int k = 0; k < kMoments; ++k) cf[k] = __shfl_sync(kFull, coef, k);
        const Real* a2 = cf + 4;
        const Real* a3 = cf + 10;
        const Real tx = a3[0] + a3[3] + a3[5], ty = a3[1] + a3[6] + a3[8], tz = a3[2] + a3[7] + a3[9];
        const Real tr2 = a2[0] + a2[3] + a2[5];
#pragma unroll
        for (int h = 0; h < (LAT::Q + 31) / 32; ++h) {
            const int q = (int)lane + 32 * h;
            if (q < LAT::Q) {
                const Real X = (Real)(R * se[3 * q]), Y = (Real)(R * se[3 * q + 1]), Z = (Real)(R * se[3 * q + 2]);
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
                a.f[(int64_t)q * a.nnodes + node] = (Real)sw[q] * sum;
            }
        }
    }
}

// LB2DSMC coefficients: one block of 64 threads per coupling cell, FP64. Each sum runs over
// the populations in lattice order: the terms (mean populations of the cell's nodes, their
// products with the speeds and with the comoving speed components) are formed in parallel,
// one population per thread, and each sum is then accumulated in order by one thread. Then
// M, C = 1 + 30 M and the new count floor(rho ppc + U).
template <typename Real, class LAT>
__global__ void __launch_bounds__(64) k_l2d_coef(MapArgs<Real> a) {
    constexpr int Q = LAT::Q;
    constexpr int NM = LAT::ORDER >= 3 ? 16 : 6;
    __shared__ double fb[Q];
    __shared__ double pj[3][Q];
    __shared__ double prod[NM][Q];
    __shared__ double s_rj[4];
    __shared__ double s_m[16];
    const uint32_t t_step = a.ctrl[CTRL_STEP];
    const int r = a.lb_ratio;
    const double rr = a.r_lat;
    const int tid = threadIdx.x;
    int e0 = 0, e1 = 0, e2 = 0;
    if (tid < Q) {
        e0 = LatTab<LAT>::e(tid, 0);
        e1 = LatTab<LAT>::e(tid, 1);
        e2 = LatTab<LAT>::e(tid, 2);
    }
    for (int ci = blockIdx.x; ci < a.n; ci += gridDim.x) {
        const int32_t cell = a.list[ci];
        if (cell < 0 || cell >= a.ncx * a.ncy) {
            if (tid == 0) {
                atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
                a.ctrl[CTRL_L2D_BAD] = 1;
            }
            continue;
        }
        const int ix = cell % a.ncx, iy = cell / a.ncx;
        if (tid < Q) {
            double sacc = 0.0;
            for (int dy = 0; dy < r; ++dy)
                for (int dx = 0; dx < r; ++dx)
                    sacc += (double)a.f[(int64_t)tid * a.nnodes + (int64_t)(iy * r + dy) * a.nx + (ix * r + dx)];
            const double fq = sacc / (double)(r * r);
            fb[tid] = fq;
            pj[0][tid] = fq * (rr * e0);
            pj[1][tid] = fq * (rr * e1);
            pj[2][tid] = fq * (rr * e2);
        }
        __syncthreads();
        if (tid < 4) {  // rho (thread 0) and rho u (threads 1-3), summed in lattice order
            const double* src = tid == 0 ? fb : pj[tid - 1];
            double acc = 0.0;
            for (int q = 0; q < Q; ++q) acc += src[q];
            s_rj[tid] = acc;
        }
        __syncthreads();
        const double rho = s_rj[0];
        const double ux = s_rj[1] / rho, uy = s_rj[2] / rho, uz = s_rj[3] / rho;
        if (tid < Q) {
            const double fq = fb[tid];
            const double c[3] = {rr * e0 - ux, rr * e1 - uy, rr * e2 - uz};
            // packed moments xx xy xz yy yz zz, xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
            prod[0][tid] = fq * c[0] * c[0];
            prod[1][tid] = fq * c[0] * c[1];
            prod[2][tid] = fq * c[0] * c[2];
            prod[3][tid] = fq * c[1] * c[1];
            prod[4][tid] = fq * c[1] * c[2];
            prod[5][tid] = fq * c[2] * c[2];
            if constexpr (NM > 6) {
                prod[6][tid] = fq * c[0] * c[0] * c[0];
                prod[7][tid] = fq * c[0] * c[0] * c[1];
                prod[8][tid] = fq * c[0] * c[0] * c[2];
                prod[9][tid] = fq * c[0] * c[1] * c[1];
                prod[10][tid] = fq * c[0] * c[1] * c[2];
                prod[11][tid] = fq * c[0] * c[2] * c[2];
                prod[12][tid] = fq * c[1] * c[1] * c[1];
                prod[13][tid] = fq * c[1] * c[1] * c[2];
                prod[14][tid] = fq * c[1] * c[2] * c[2];
                prod[15][tid] = fq * c[2] * c[2] * c[2];
            }
        }
        __syncthreads();
        if (tid < NM) {
            double acc = 0.0;
            for (int q = 0; q < Q; ++q) acc += prod[tid][q];
            double v = acc / rho;
            if (tid == 0 || tid == 3 || tid == 5) v -= 1.0;
            s_m[tid] = v;
        }
        __syncthreads();
        if (tid == 0) {
            GradRec g;
            g.rho = rho;
            g.u[0] = ux;
            g.u[1] = uy;
            g.u[2] = uz;
            double M = 0.0;
            for (int k = 0; k < 6; ++k) {
                g.a2[k] = s_m[k];
                M = fmax(M, fabs(s_m[k]));
            }
            for (int k = 0; k < 10; ++k) {
                g.a3[k] = NM > 6 ? s_m[6 + k] : 0.0;
                M = fmax(M, fabs(g.a3[k]));
            }
            g.C = 1.0 + 30.0 * M;
            const double u = u01d(draw(a.seed, (uint32_t)cell, t_step, TAG_L2D_ROUND, 0, 0).x);
            const double ne = floor(rho * (double)a.ppc + u);
            g.nnew = ne > 0.0 ? (uint32_t)ne : 0u;
            g.pad = 0;
            a.grad[ci] = g;
        }
        __syncthreads();
    }
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

constexpr int kSampleWarps = 4;

// One block per coupling cell: the cell's trial stream is evaluated 128 trials at a time;
// the k-th accepted trial becomes the k-th particle of the cell's bin, replacing the old
// ones. Nothing is written if a listed cell index was invalid (the coefficient kernel
// flagged it).
template <typename Real, class LAT>
__global__ void __launch_bounds__(kSampleWarps * 32) k_l2d_sample(MapArgs<Real> a) {
    __shared__ unsigned s_am[kSampleWarps], s_em[kSampleWarps], s_vm[kSampleWarps];
    if (a.ctrl[CTRL_L2D_BAD]) return;
    const uint32_t t_step = a.ctrl[CTRL_STEP];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int w = threadIdx.x >> 5;
    const uint32_t bin = (uint32_t)a.bin;
    unsigned long long deleted = 0, created = 0, attempts = 0, envelope = 0;
    uint32_t flags = 0;
    int32_t dlive = 0;
    for (int ci = blockIdx.x; ci < a.n; ci += gridDim.x) {
        const uint32_t cell = (uint32_t)a.list[ci];
        const GradRec& g = a.grad[ci];
        const uint32_t nnew = g.nnew;
        if (nnew > bin) {  // the cell keeps its particles
            flags |= HYB_ST_CAPACITY;
            continue;
        }
        Real a2[6], a3[10];
#pragma unroll
        for (int k = 0; k < 6; ++k) a2[k] = (Real)g.a2[k];
#pragma unroll
        for (int k = 0; k < 10; ++k) a3[k] = (Real)g.a3[k];
        const Real C = (Real)g.C;
        const Real ux = (Real)g.u[0], uy = (Real)g.u[1], uz = (Real)g.u[2];
        const int64_t out0 = (int64_t)cell * bin;
        const Real fx = (Real)(cell % (uint32_t)a.ncx), fy = (Real)(cell / (uint32_t)a.ncx);
        const uint64_t cap64 = 1000ull * nnew;
        const uint32_t cap = cap64 < 0xFFFFFFull ? (uint32_t)cap64 : 0xFFFFFFu;
        uint32_t produced = 0, j0 = 0;
        while (produced < nnew && j0 < cap) {
            const uint32_t j = j0 + threadIdx.x;
            const bool valid = j < cap;
            bool acc = false, env = false;
            Real X = 0, Y = 0, Z = 0;
            uint4 r2 = make_uint4(0, 0, 0, 0);
            if (valid) {
                const uint4 r1 = draw(a.seed, cell, t_step, TAG_L2D_VEL, j, 0);
                r2 = draw(a.seed, cell, t_step, TAG_L2D_VEL, j, 1);
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
            for (int v = 0; v < kSampleWarps; ++v) {
                const uint32_t cv = (uint32_t)__popc(s_am[v]);
                if (v < w) before += cv;
                total += cv;
            }
            const uint32_t need = nnew - produced;
            const uint32_t rank = before + (uint32_t)__popc(am & lt);
            if (acc && rank < need) {
                const int64_t slot = out0 + produced + rank;
                a.x[slot] = fx + (Real)u01f(r2.y);
                a.y[slot] = fy + (Real)u01f(r2.z);
                a.vx[slot] = X + ux;
                a.vy[slot] = Y + uy;
                a.vz[slot] = Z + uz;
            }
            if (threadIdx.x == 0) {
                // trials consumed this round: up to the need-th accepted one, or all valid ones
                uint32_t used = 0, envc = 0;
                if (total >= need) {
                    uint32_t left = need;
                    for (int v = 0; v < kSampleWarps; ++v) {
                        const uint32_t cv = (uint32_t)__popc(s_am[v]);
                        if (left > cv) {
                            left -= cv;
                            used += 32;
                            envc += (uint32_t)__popc(s_em[v] & s_vm[v]);
                            continue;
                        }
                        int bit = 0;
                        for (unsigned mm = s_am[v];; mm &= mm - 1u) {
                            bit = __ffs(mm) - 1;
                            if (--left == 0) break;
                        }
                        const unsigned upto = bit == 31 ? 0xFFFFFFFFu : ((2u << bit) - 1u);
                        used += (uint32_t)bit + 1u;
                        envc += (uint32_t)__popc(s_em[v] & upto);
                        break;
                    }
                } else {
                    for (int v = 0; v < kSampleWarps; ++v) {
                        used += (uint32_t)__popc(s_vm[v]);
                        envc += (uint32_t)__popc(s_em[v] & s_vm[v]);
                    }
                }
                attempts += used;
                envelope += envc;
            }
            produced += min(total, need);
            j0 += kSampleWarps * 32;
            __syncthreads();
        }
        if (produced < nnew) flags |= HYB_ST_SAMPLING_CAP;
        if (threadIdx.x == 0) {
            const uint32_t old = a.count[cell];
            deleted += old;
            created += produced;
            dlive += (int32_t)produced - (int32_t)old;
            a.count[cell] = produced;
        }
    }
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
    a.r_lat = c.d.r_lat;
    a.seed = c.p.seed;
    a.acc = c.st.acc;
    a.ctrl = c.st.ctrl;
    a.counters = c.st.counters;
    a.grad = c.st.grad;
    a.count = c.st.count[c.cur_p];
    a.x = (Real*)c.st.px[c.cur_p];
    a.y = (Real*)c.st.py[c.cur_p];
    a.vx = (Real*)c.st.pvx[c.cur_p];
    a.vy = (Real*)c.st.pvy[c.cur_p];
    a.vz = (Real*)c.st.pvz[c.cur_p];
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
    k_d2l<Real, LAT><<<blocks_for(c, (int64_t)n * 32, 128, 16), 128, 0, c.stream>>>(a);
    prof_end(c, K_D2L);
    return cudaGetLastError();
}

template <typename Real, class LAT>
cudaError_t l2d_impl(Ctx& c, const int32_t* cells, int32_t n) {
    MapArgs<Real> a = map_args<Real>(c, cells, n);
    cudaError_t e = cudaMemsetAsync(c.st.ctrl + CTRL_L2D_BAD, 0, 4, c.stream);
    if (e != cudaSuccess) return e;
    prof_begin(c, K_L2D_COEF);
    k_l2d_coef<Real, LAT><<<blocks_for(c, (int64_t)n * 64, 64, 32), 64, 0, c.stream>>>(a);
    prof_end(c, K_L2D_COEF);
    prof_begin(c, K_L2D_SAMPLE);
    k_l2d_sample<Real, LAT><<<blocks_for(c, (int64_t)n * 32 * kSampleWarps, 32 * kSampleWarps, 16),
                              32 * kSampleWarps, 0, c.stream>>>(a);
    prof_end(c, K_L2D_SAMPLE);
    return cudaGetLastError();
}

constexpr int kMaxDevices = 64;
GradRec* g_scratch_addr[kMaxDevices] = {};

// Device address of the fixed scratch on `device`, which must be the current device.
cudaError_t noalloc_scratch(int device, GradRec** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_l2d_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = (GradRec*)p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

template <typename Real, class LAT>
cudaError_t l2d_noalloc_impl(Ctx& c, const int32_t* cells, int32_t n, GradRec* rec) {
    MapArgs<Real> a = map_args<Real>(c, cells, n);
    a.grad = rec;  // the fixed array instead of the arena's records
    cudaError_t e = cudaMemsetAsync(c.st.ctrl + CTRL_L2D_BAD, 0, 4, c.stream);
    if (e != cudaSuccess) return e;
    prof_begin(c, K_L2D_COEF);
    k_l2d_coef<Real, LAT><<<blocks_for(c, (int64_t)n * 64, 64, 32), 64, 0, c.stream>>>(a);
    prof_end(c, K_L2D_COEF);
    prof_begin(c, K_L2D_SAMPLE);
    k_l2d_sample<Real, LAT><<<blocks_for(c, (int64_t)n * 32 * kSampleWarps, 32 * kSampleWarps, 16),
                              32 * kSampleWarps, 0, c.stream>>>(a);
    prof_end(c, K_L2D_SAMPLE);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_map_l2d_noalloc(Ctx& c, const int32_t* cells, int32_t n) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != c.device) return cudaErrorInvalidDevice;
    GradRec* rec = nullptr;
    e = noalloc_scratch(dev, &rec);
    if (e != cudaSuccess) return e;
    if (c.p.lattice == 39)
        return c.p.real_bytes == 4 ? l2d_noalloc_impl<float, D3Q39>(c, cells, n, rec)
                                   : l2d_noalloc_impl<double, D3Q39>(c, cells, n, rec);
    return c.p.real_bytes == 4 ? l2d_noalloc_impl<float, D3Q19>(c, cells, n, rec)
                               : l2d_noalloc_impl<double, D3Q19>(c, cells, n, rec);
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
