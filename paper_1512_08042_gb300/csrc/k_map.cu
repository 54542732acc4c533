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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

template <typename Real, class LAT>
__global__ void __launch_bounds__(128) k_d2l(MapArgs<Real> a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const int32_t node = a.list[t];
    if (node < 0 || (int64_t)node >= a.nnodes) {
        atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
        return;
    }
    const int x = node % a.nx, y = node / a.nx;
    const int64_t cell = (int64_t)(y / a.lb_ratio) * a.ncx + (x / a.lb_ratio);
    const uint32_t S = a.ctrl[CTRL_NSAMPLES];
    const double* m = a.acc + cell * kMoments;
    const double NS = m[0];
    if (S == 0 || !(NS > 0.0)) {
        atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
        return;
    }
    // FP64 coefficient solve
    const double rho = (NS / (double)S) / (double)a.ppc;
    const double iNS = 1.0 / NS;
    const double m1x = m[1] * iNS, m1y = m[2] * iNS, m1z = m[3] * iNS;
    const double d2[6] = {1, 0, 0, 1, 0, 1};
    // sym(<v> I) for the packed entries xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    const double s3[10] = {3 * m1x, m1y, m1z, m1x, 0.0, m1x, 3 * m1y, m1z, m1y, 3 * m1z};
    Real a2[6], a3[10];
    for (int k = 0; k < 6; ++k) a2[k] = (Real)(rho * (m[4 + k] * iNS - d2[k]));
    for (int k = 0; k < 10; ++k) a3[k] = (Real)(rho * (m[10 + k] * iNS - s3[k]));
    const Real r0 = (Real)rho, a1x = (Real)(rho * m1x), a1y = (Real)(rho * m1y), a1z = (Real)(rho * m1z);
    const Real tx = a3[0] + a3[3] + a3[5], ty = a3[1] + a3[6] + a3[8], tz = a3[2] + a3[7] + a3[9];
    const Real tr2 = a2[0] + a2[3] + a2[5];
    constexpr double R = lat_r<LAT>();
#pragma unroll
    for (int q = 0; q < LAT::Q; ++q) {
        const Real X = (Real)(R * E<LAT>(q, 0)), Y = (Real)(R * E<LAT>(q, 1)), Z = (Real)(R * E<LAT>(q, 2));
        const Real h2 = a2[0] * X * X + a2[3] * Y * Y + a2[5] * Z * Z - tr2 +
                        (Real)2 * (a2[1] * X * Y + a2[2] * X * Z + a2[4] * Y * Z);
        Real sum = r0 + a1x * X + a1y * Y + a1z * Z + (Real)0.5 * h2;
        if (LAT::ORDER >= 3) {
            const Real cubic = a3[0] * X * X * X + (Real)3 * a3[1] * X * X * Y + (Real)3 * a3[2] * X * X * Z +
                               (Real)3 * a3[3] * X * Y * Y + (Real)6 * a3[4] * X * Y * Z +
                               (Real)3 * a3[5] * X * Z * Z + a3[6] * Y * Y * Y + (Real)3 * a3[7] * Y * Y * Z +
                               (Real)3 * a3[8] * Y * Z * Z + a3[9] * Z * Z * Z;
            sum += (cubic - (Real)3 * (tx * X + ty * Y + tz * Z)) * (Real)(1.0 / 6.0);
        }
        a.f[(int64_t)q * a.nnodes + node] = (Real)LatTab<LAT>::w(q) * sum;
    }
}

// One warp per coupling cell: FP64 Grad coefficients and the particle count.
template <typename Real, class LAT>
__global__ void __launch_bounds__(64) k_l2d_coef(MapArgs<Real> a) {
    const uint32_t t_step = a.ctrl[CTRL_STEP];
    const int r = a.lb_ratio;
    const double rr = a.r_lat;
    const unsigned lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    constexpr int QL = (LAT::Q + 31) / 32;
    for (int ci = gw; ci < a.n; ci += nw) {
        const int32_t cell = a.list[ci];
        if (cell < 0 || cell >= a.ncx * a.ncy) {
            if (lane == 0) {
                atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
                a.ctrl[CTRL_L2D_BAD] = 1;
            }
            continue;
        }
        const int ix = cell % a.ncx, iy = cell / a.ncx;
        double fb[QL];
        double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int h = 0; h < QL; ++h) {
            const int q = lane + 32 * h;
            double s = 0.0;
            if (q < LAT::Q) {
                for (int dy = 0; dy < r; ++dy)
                    for (int dx = 0; dx < r; ++dx)
                        s += (double)a.f[(int64_t)q * a.nnodes + (int64_t)(iy * r + dy) * a.nx + (ix * r + dx)];
                s = s / (double)(r * r);
                rho += s;
                jx += s * (rr * LatTab<LAT>::e(q, 0));
                jy += s * (rr * LatTab<LAT>::e(q, 1));
                jz += s * (rr * LatTab<LAT>::e(q, 2));
            }
            fb[h] = s;
        }
        rho = warp_sum(rho);
        const double irho = 1.0 / rho;
        const double ux = warp_sum(jx) * irho, uy = warp_sum(jy) * irho, uz = warp_sum(jz) * irho;
        double m2[6] = {0, 0, 0, 0, 0, 0}, m3[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int h = 0; h < QL; ++h) {
            const int q = lane + 32 * h;
            if (q < LAT::Q) {
                const double cx = rr * LatTab<LAT>::e(q, 0) - ux;
                const double cy = rr * LatTab<LAT>::e(q, 1) - uy;
                const double cz = rr * LatTab<LAT>::e(q, 2) - uz;
                const double f = fb[h];
                m2[0] += f * cx * cx * irho;
                m2[1] += f * cx * cy * irho;
                m2[2] += f * cx * cz * irho;
                m2[3] += f * cy * cy * irho;
                m2[4] += f * cy * cz * irho;
                m2[5] += f * cz * cz * irho;
                if (LAT::ORDER >= 3) {
                    m3[0] += f * cx * cx * cx * irho;
                    m3[1] += f * cx * cx * cy * irho;
                    m3[2] += f * cx * cx * cz * irho;
                    m3[3] += f * cx * cy * cy * irho;
                    m3[4] += f * cx * cy * cz * irho;
                    m3[5] += f * cx * cz * cz * irho;
                    m3[6] += f * cy * cy * cy * irho;
                    m3[7] += f * cy * cy * cz * irho;
                    m3[8] += f * cy * cz * cz * irho;
                    m3[9] += f * cz * cz * cz * irho;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) m2[k] = warp_sum(m2[k]);
        if (LAT::ORDER >= 3) {
#pragma unroll
            for (int k = 0; k < 10; ++k) m3[k] = warp_sum(m3[k]);
        }
        if (lane == 0) {
            GradRec g;
            g.rho = rho;
            g.u[0] = ux;
            g.u[1] = uy;
            g.u[2] = uz;
            for (int k = 0; k < 6; ++k) g.a2[k] = m2[k];
            g.a2[0] -= 1.0;
            g.a2[3] -= 1.0;
            g.a2[5] -= 1.0;
            for (int k = 0; k < 10; ++k) g.a3[k] = m3[k];
            double M = 0.0;
            for (int k = 0; k < 6; ++k) M = fmax(M, fabs(g.a2[k]));
            for (int k = 0; k < 10; ++k) M = fmax(M, fabs(g.a3[k]));
            g.C = 1.0 + 30.0 * M;
            const double u = u01d(draw(a.seed, (uint32_t)cell, t_step, TAG_L2D_ROUND, 0, 0).x);
            const double ne = floor(rho * (double)a.ppc + u);
            g.nnew = ne > 0.0 ? (uint32_t)ne : 0u;
            g.pad = 0;
            a.grad[ci] = g;
        }
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

// One warp per coupling cell: the cell's trial stream is evaluated 32 trials at a time; the
// k-th accepted trial becomes the k-th particle of the cell's bin, replacing the old ones.
// Nothing is written if a listed cell index was invalid (the coefficient kernel flagged it).
template <typename Real, class LAT>
__global__ void __launch_bounds__(64) k_l2d_sample(MapArgs<Real> a) {
    if (a.ctrl[CTRL_L2D_BAD]) return;
    const uint32_t t_step = a.ctrl[CTRL_STEP];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t bin = (uint32_t)a.bin;
    unsigned long long deleted = 0, created = 0, attempts = 0, envelope = 0;
    uint32_t flags = 0;
    int32_t dlive = 0;
    for (int ci = gw; ci < a.n; ci += nw) {
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
            const uint32_t j = j0 + lane;
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
            const unsigned amask = __ballot_sync(kFull, acc);
            const unsigned emask = __ballot_sync(kFull, env);
            const unsigned vmask = __ballot_sync(kFull, valid);
            const uint32_t need = nnew - produced;
            const uint32_t rank = __popc(amask & lt);
            uint32_t used_mask = vmask;  // trials consumed this round
            if ((uint32_t)__popc(amask) >= need) {
                const unsigned lastm = __ballot_sync(kFull, acc && rank == need - 1u);
                const int last = __ffs(lastm) - 1;
                used_mask = last == 31 ? 0xFFFFFFFFu : ((2u << last) - 1u);
            }
            if (acc && rank < need) {
                const int64_t slot = out0 + produced + rank;
                a.x[slot] = fx + (Real)u01f(r2.y);
                a.y[slot] = fy + (Real)u01f(r2.z);
                a.vx[slot] = X + ux;
                a.vy[slot] = Y + uy;
                a.vz[slot] = Z + uz;
            }
            if (lane == 0) {
                attempts += (unsigned long long)__popc(used_mask);
                envelope += (unsigned long long)__popc(emask & used_mask);
            }
            produced += min((uint32_t)__popc(amask), need);
            j0 += 32;
        }
        if (produced < nnew) flags |= HYB_ST_SAMPLING_CAP;
        if (lane == 0) {
            const uint32_t old = a.count[cell];
            deleted += old;
            created += produced;
            dlive += (int32_t)produced - (int32_t)old;
            a.count[cell] = produced;
        }
    }
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0) {
        if (deleted) atomicAdd(&a.counters[HYB_C_DELETED], deleted);
        if (created) atomicAdd(&a.counters[HYB_C_CREATED], created);
        if (attempts) atomicAdd(&a.counters[HYB_C_L2D_ATTEMPTS], attempts);
        if (envelope) atomicAdd(&a.counters[HYB_C_ENVELOPE], envelope);
        if (dlive) atomicAdd(&a.ctrl[CTRL_NTOT], (uint32_t)dlive);
        if (flags) atomicOr(&a.ctrl[CTRL_STATUS], flags);
    }
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
    k_d2l<Real, LAT><<<(n + 127) / 128, 128, 0, c.stream>>>(a);
    prof_end(c, K_D2L);
    return cudaGetLastError();
}

template <typename Real, class LAT>
cudaError_t l2d_impl(Ctx& c, const int32_t* cells, int32_t n) {
    MapArgs<Real> a = map_args<Real>(c, cells, n);
    cudaError_t e = cudaMemsetAsync(c.st.ctrl + CTRL_L2D_BAD, 0, 4, c.stream);
    if (e != cudaSuccess) return e;
    prof_begin(c, K_L2D_COEF);
    k_l2d_coef<Real, LAT><<<blocks_for(c, (int64_t)n * 32, 64, 32), 64, 0, c.stream>>>(a);
    prof_end(c, K_L2D_COEF);
    prof_begin(c, K_L2D_SAMPLE);
    k_l2d_sample<Real, LAT><<<blocks_for(c, (int64_t)n * 32, 64, 32), 64, 0, c.stream>>>(a);
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
    k_l2d_coef<Real, LAT><<<blocks_for(c, (int64_t)n * 32, 64, 32), 64, 0, c.stream>>>(a);
    prof_end(c, K_L2D_COEF);
    prof_begin(c, K_L2D_SAMPLE);
    k_l2d_sample<Real, LAT><<<blocks_for(c, (int64_t)n * 32, 64, 32), 64, 0, c.stream>>>(a);
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
