// The two kinetic mappings of Sec. 2, in FP64 arithmetic with Real (float or double) state.
//
// k_d2l (DSMC2LB, Sec. 2.1): one thread per coupling node. The cumulative sums of the
// node's DSMC cell give rho = <N>/ppc, the per-particle raw moments <v>, <vv>, <vvv>, and
// the raw Hermite coefficients a0 = rho, a1 = rho <v>, a2 = rho(<vv> - I),
// a3 = rho(<vvv> - sym(<v> I)); the populations are f_a = w_a sum_{n<=N} a^(n):H^(n)(xi_a)/n!
// (Eq. discretefunctions).
//
// k_l2d_prep + k_l2d_sample (LB2DSMC, Sec. 2.2, Table 1): the first (one block) computes per
// coupling cell the mean populations of its lb_ratio^2 nodes, rho and u, the comoving
// coefficients a2 = sum f c c / rho - I and a3 = sum f c c c / rho (c = xi - u), M, C = 1 + 30 M
// (Eq. C), the particle count floor(rho ppc + U), and the append offsets (a block scan);
// the second (one warp per cell) marks the cell's old particles deleted and draws the new
// ones: Box-Muller trial xi from the unit Maxwellian, accepted when C R <= G(xi) with
// G = 1 + a2:H2/2 + a3:H3/6 (Eq. distr_outeq), velocity xi + u (Eq. step6 in c_th units),
// position uniform in the cell. Draws are keyed by (cell, step, purpose, particle index,
// trial), so the result does not depend on the launch shape.
#include "hyb_internal.cuh"

namespace hyb {

namespace {

template <class LAT>
__host__ __device__ constexpr int E(int a, int i) {
    return LatTab<LAT>::e(a, i);
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
    const double rho = (NS / (double)S) / (double)a.ppc;
    const double m1x = m[1] / NS, m1y = m[2] / NS, m1z = m[3] / NS;
    double a2[6], a3[10];
    const double d2[6] = {1, 0, 0, 1, 0, 1};
    for (int k = 0; k < 6; ++k) a2[k] = rho * (m[4 + k] / NS - d2[k]);
    // sym(<v> I) for the packed entries xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    const double s3[10] = {3 * m1x, m1y, m1z, m1x, 0.0, m1x, 3 * m1y, m1z, m1y, 3 * m1z};
    for (int k = 0; k < 10; ++k) a3[k] = rho * (m[10 + k] / NS - s3[k]);
    const double a1x = rho * m1x, a1y = rho * m1y, a1z = rho * m1z;
    const double r = a.r_lat;
#pragma unroll
    for (int q = 0; q < LAT::Q; ++q) {
        const double xi[3] = {r * E<LAT>(q, 0), r * E<LAT>(q, 1), r * E<LAT>(q, 2)};
        double s = rho + a1x * xi[0] + a1y * xi[1] + a1z * xi[2] + 0.5 * herm2_contract(a2, xi);
        if (LAT::ORDER >= 3) s += herm3_contract(a3, xi) / 6.0;
        a.f[(int64_t)q * a.nnodes + node] = (Real)(LatTab<LAT>::w(q) * s);
    }
}

template <typename Real, class LAT>
__global__ void __launch_bounds__(256) k_l2d_prep(MapArgs<Real> a) {
    __shared__ uint32_t warp_tot[8];
    __shared__ uint32_t s_carry;
    const uint32_t t_step = a.ctrl[CTRL_STEP];
    const int r = a.lb_ratio;
    const double rr = a.r_lat;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    int bad = 0;
    __syncthreads();
    for (int base = 0; base < a.n; base += blockDim.x) {
        const int ci = base + threadIdx.x;
        uint32_t nn = 0;
        if (ci < a.n) {
            const int32_t cell = a.list[ci];
            if (cell < 0 || cell >= a.ncx * a.ncy) {
                bad = 1;
            } else {
                const int ix = cell % a.ncx, iy = cell / a.ncx;
                double fb[LAT::Q];
                double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
                for (int q = 0; q < LAT::Q; ++q) {
                    double s = 0.0;
                    for (int dy = 0; dy < r; ++dy)
                        for (int dx = 0; dx < r; ++dx)
                            s += (double)a.f[(int64_t)q * a.nnodes + (int64_t)(iy * r + dy) * a.nx +
                                             (ix * r + dx)];
                    fb[q] = s / (double)(r * r);
                }
#pragma unroll
                for (int q = 0; q < LAT::Q; ++q) {
                    rho += fb[q];
                    jx += fb[q] * (rr * E<LAT>(q, 0));
                    jy += fb[q] * (rr * E<LAT>(q, 1));
                    jz += fb[q] * (rr * E<LAT>(q, 2));
                }
                GradRec g;
                g.rho = rho;
                g.u[0] = jx / rho;
                g.u[1] = jy / rho;
                g.u[2] = jz / rho;
                for (int k = 0; k < 6; ++k) g.a2[k] = 0.0;
                for (int k = 0; k < 10; ++k) g.a3[k] = 0.0;
#pragma unroll
                for (int q = 0; q < LAT::Q; ++q) {
                    const double cx = rr * E<LAT>(q, 0) - g.u[0];
                    const double cy = rr * E<LAT>(q, 1) - g.u[1];
                    const double cz = rr * E<LAT>(q, 2) - g.u[2];
                    const double f = fb[q];
                    g.a2[0] += f * cx * cx / rho;
                    g.a2[1] += f * cx * cy / rho;
                    g.a2[2] += f * cx * cz / rho;
                    g.a2[3] += f * cy * cy / rho;
                    g.a2[4] += f * cy * cz / rho;
                    g.a2[5] += f * cz * cz / rho;
                    if (LAT::ORDER >= 3) {
                        g.a3[0] += f * cx * cx * cx / rho;
                        g.a3[1] += f * cx * cx * cy / rho;
                        g.a3[2] += f * cx * cx * cz / rho;
                        g.a3[3] += f * cx * cy * cy / rho;
                        g.a3[4] += f * cx * cy * cz / rho;
                        g.a3[5] += f * cx * cz * cz / rho;
                        g.a3[6] += f * cy * cy * cy / rho;
                        g.a3[7] += f * cy * cy * cz / rho;
                        g.a3[8] += f * cy * cz * cz / rho;
                        g.a3[9] += f * cz * cz * cz / rho;
                    }
                }
                g.a2[0] -= 1.0;
                g.a2[3] -= 1.0;
                g.a2[5] -= 1.0;
                double M = 0.0;
                for (int k = 0; k < 6; ++k) M = fmax(M, fabs(g.a2[k]));
                for (int k = 0; k < 10; ++k) M = fmax(M, fabs(g.a3[k]));
                g.C = 1.0 + 30.0 * M;
                const double u = u01d(draw(a.seed, (uint32_t)cell, t_step, TAG_L2D_ROUND, 0, 0).x);
                const double ne = floor(rho * (double)a.ppc + u);
                nn = ne > 0.0 ? (uint32_t)ne : 0u;
                g.nnew = nn;
                g.offset = 0;
                a.grad[ci] = g;
            }
        }
        // block exclusive scan of nn
        uint32_t incl = nn;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t yv = __shfl_up_sync(kFull, incl, off);
            if ((int)lane >= off) incl += yv;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            if (i < w) wpre += warp_tot[i];
            tot += warp_tot[i];
        }
        const uint32_t carry = s_carry;
        if (ci < a.n) a.grad[ci].offset = carry + wpre + incl - nn;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    const int any_bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        const uint32_t total = s_carry;
        const uint32_t base = a.ctrl[CTRL_NTOT];
        if (any_bad) {
            atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_BAD_INPUT);
            a.ctrl[CTRL_L2D_SKIP] = 1;
        } else if ((int64_t)base + total > a.capacity) {
            atomicOr(&a.ctrl[CTRL_STATUS], HYB_ST_CAPACITY);
            a.ctrl[CTRL_L2D_SKIP] = 1;
        } else {
            a.ctrl[CTRL_L2D_SKIP] = 0;
            a.ctrl[CTRL_L2D_BASE] = base;
            a.ctrl[CTRL_NTOT] = base + total;
            atomicAdd(&a.counters[HYB_C_CREATED], (unsigned long long)total);
        }
    }
}

template <typename Real, class LAT>
__global__ void __launch_bounds__(128) k_l2d_sample(MapArgs<Real> a) {
    if (a.ctrl[CTRL_L2D_SKIP]) return;
    const uint32_t base = a.ctrl[CTRL_L2D_BASE];
    const uint32_t t_step = a.ctrl[CTRL_STEP];
    const unsigned lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long deleted = 0, attempts = 0, envelope = 0;
    uint32_t flags = 0;
    for (int ci = gw; ci < a.n; ci += nw) {
        const uint32_t cell = (uint32_t)a.list[ci];
        const GradRec g = a.grad[ci];
        const uint32_t s0 = a.cell_start[cell], s1 = a.cell_start[cell + 1];
        for (uint32_t i = s0 + lane; i < s1; i += 32) {
            if (a.x[i] >= (Real)0) deleted += 1;
            a.x[i] = (Real)-1;
        }
        const int ix = (int)(cell % (uint32_t)a.ncx), iy = (int)(cell / (uint32_t)a.ncx);
        for (uint32_t k = lane; k < g.nnew; k += 32) {
            const uint4 rp = draw(a.seed, cell, t_step, TAG_L2D_POS, k, 0);
            double v[3] = {g.u[0], g.u[1], g.u[2]};
            int att = 0;
            bool done = false;
            for (; att < kMaxL2DAttempts && !done; ++att) {
                const uint4 r1 = draw(a.seed, cell, t_step, TAG_L2D_VEL, k, (uint32_t)(2 * att));
                const uint4 r2 = draw(a.seed, cell, t_step, TAG_L2D_VEL, k, (uint32_t)(2 * att + 1));
                double n0, n1, n2, n3;
                box_muller(r1.x, r1.y, n0, n1);
                box_muller(r1.z, r1.w, n2, n3);
                const double xd[3] = {(double)(Real)n0, (double)(Real)n1, (double)(Real)n2};
                double G = 1.0 + 0.5 * herm2_contract(g.a2, xd);
                if (LAT::ORDER >= 3) G += herm3_contract(g.a3, xd) / 6.0;
                const double R = u01d(r2.x);
                if (G > g.C) envelope += 1;
                if (g.C * R <= G) {
                    v[0] = xd[0] + g.u[0];
                    v[1] = xd[1] + g.u[1];
                    v[2] = xd[2] + g.u[2];
                    done = true;
                }
            }
            if (!done) flags |= HYB_ST_SAMPLING_CAP;
            attempts += (unsigned long long)att;
            const uint32_t slot = base + g.offset + k;
            a.x[slot] = (Real)ix + (Real)u01f(rp.x);
            a.y[slot] = (Real)iy + (Real)u01f(rp.y);
            a.vx[slot] = (Real)v[0];
            a.vy[slot] = (Real)v[1];
            a.vz[slot] = (Real)v[2];
        }
    }
    deleted = __reduce_add_sync(kFull, (unsigned)deleted);
    attempts = __reduce_add_sync(kFull, (unsigned)attempts);
    envelope = __reduce_add_sync(kFull, (unsigned)envelope);
    flags = __reduce_or_sync(kFull, flags);
    if (lane == 0) {
        if (deleted) atomicAdd(&a.counters[HYB_C_DELETED], deleted);
        if (attempts) atomicAdd(&a.counters[HYB_C_L2D_ATTEMPTS], attempts);
        if (envelope) atomicAdd(&a.counters[HYB_C_ENVELOPE], envelope);
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
    a.nnodes = c.d.nnodes;
    a.capacity = c.d.capacity;
    a.list = list;
    a.r_lat = c.d.r_lat;
    a.seed = c.p.seed;
    a.acc = c.st.acc;
    a.ctrl = c.st.ctrl;
    a.counters = c.st.counters;
    a.grad = c.st.grad;
    a.cell_start = c.st.cell_start;
    a.x = (Real*)c.st.px[c.cur_p];
    a.y = (Real*)c.st.py[c.cur_p];
    a.vx = (Real*)c.st.pvx[c.cur_p];
    a.vy = (Real*)c.st.pvy[c.cur_p];
    a.vz = (Real*)c.st.pvz[c.cur_p];
    return a;
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
    prof_begin(c, K_L2D_PREP);
    k_l2d_prep<Real, LAT><<<1, 256, 0, c.stream>>>(a);
    prof_end(c, K_L2D_PREP);
    int64_t blocks = ((int64_t)n * 32 + 127) / 128;
    if (blocks > (int64_t)c.num_sms * 16) blocks = (int64_t)c.num_sms * 16;
    prof_begin(c, K_L2D_SAMPLE);
    k_l2d_sample<Real, LAT><<<(unsigned)blocks, 128, 0, c.stream>>>(a);
    prof_end(c, K_L2D_SAMPLE);
    return cudaGetLastError();
}

}  // namespace

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
