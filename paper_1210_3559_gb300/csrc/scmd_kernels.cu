// scmd_kernels.cu -- sm_103a kernels of the Sutton-Chen cluster MD hot path.
//
// Per MD step two pair passes run, the paper's "two successive two-body
// problems" (Sec. II, "Computational approach"):
//   density pass  rho_i = a^m sum_{j!=i} r_ij^-m                      (Eq. 2)
//   force pass    F_i = sum_{j!=i} r_ij^-2 [A r_ij^-n - B (g_i + g_j) r_ij^-m] (r_i - r_j)
//                 with A = eps n a^n, B = eps c m/2 a^m, g = rho^-1/2  (-dU/dr of Eq. 1)
// and the force pass's epilogue finishes the velocity-Verlet step and starts the
// next one (BAOAB Langevin, NVE, or the Berendsen split) for the atoms it owns.
//
// Work decomposition of a pair pass (no tensor cores: the work is FP32 SIMT
// arithmetic plus one MUFU reciprocal / reciprocal square root per pair):
//   * a work item is an i-block of 32*IPT atoms of one cluster; each thread
//     keeps IPT i-atoms in registers;
//   * the item's j-range (all atoms of the cluster, in 32-atom tiles) is split
//     over the W warps of a CTA and the C CTAs of a thread-block cluster; each
//     warp stages its own j-tile in shared memory with one coalesced 16-byte
//     load per lane and reads it back with broadcast loads;
//   * per-thread partial sums are reduced over warps in shared memory and over
//     the CTAs of the cluster through distributed shared memory, in a fixed
//     order (results are run-to-run deterministic); the cluster's rank-0 CTA
//     owns the epilogue.
// Precision (MIXED): pair terms in FP32 on FP32 coordinates relative to a fixed
// per-cluster origin near the centre of mass; each
// 32-pair tile is summed in FP32, tiles are summed in FP32 spans of 4 tiles,
// spans are folded into FP64 (density, energy) or into FP32 running sums
// (forces); reductions over warps/CTAs are FP64 (density, energy) or FP32
// (forces); positions and velocities are integrated in FP64.
// Precision (FP64): every operation in IEEE double.
#include "scmd_device.cuh"

namespace scmd {
// The j-range of an item is split over the warps of its thread-block cluster in units of
// 32 / kSplit<PREC> atoms. FP32 passes use whole 32-atom tiles. FP64 passes use 4-atom units: an FP64
// warp instruction occupies an SM sub-partition's FP64 pipe for ~68 cycles on this part, so a whole
// tile of pairs is ~20 us of one warp's work, and a small cluster (a few tiles) needs finer units to
// spread over more warps.
template <int PREC> struct SplitOf;
template <> struct SplitOf<1> { static constexpr int S = 1; };
template <> struct SplitOf<0> { static constexpr int S = 8; };

// ------------------------------------------------------------- density pass
// Shared memory: tiles [W][32] V4 | red [W][BI] double | inbox [C][BI] double (read on rank 0)
template <int PREC, int IPT, int SPECIAL, int CUT>
__global__ void __launch_bounds__(512, (PREC == 1 && IPT < 4) ? 2 : 1) k_density(const Dev d, const Item* __restrict__ items, int C, int obs) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    constexpr int BI = 32 * IPT;
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_bar;  // rank 0: completes when the other ranks' partials have landed
    __shared__ int s_late;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    if (rank == 0 && threadIdx.x == 0) mbar_setup(&s_bar, (unsigned)((C - 1) * BI * 8));
    cluster_arrive_relaxed();  // "this CTA has started": waited for before any remote store
    pdl_launch_dependents();
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Item it = load_item<BI>(d, items, C);
    V4* tiles = reinterpret_cast<V4*>(smem);
    // MIXED: partials are double-float (2 floats); FP64: one double (same 8 bytes)
    double* red = reinterpret_cast<double*>(smem + (size_t)W * 32 * sizeof(V4));
    double* inbox = red + W * BI;
    f2sum* red2 = reinterpret_cast<f2sum*>(red);
    f2sum* inbox2 = reinterpret_cast<f2sum*>(inbox);
    const V4* mir = reinterpret_cast<const V4*>(d.mirror);
    const R rc2 = PREC == 1 ? (R)d.pot.rcut2f : (R)d.pot.rcut2;  // no FP64 conversion in MIXED
    const int mexp = d.pot.m;
    constexpr int S = SplitOf<PREC>::S, L = 32 / S;
    const int ntile = (it.nj + 31) >> 5, nunit = ntile * S;
    const int Q = C * W, qi = rank * W + warp;
    const int u_beg = (int)(((long long)nunit * qi) / Q), u_end = (int)(((long long)nunit * (qi + 1)) / Q);
    const int t_last = (u_end - 1) / S;  // last tile this warp touches
    const int tdiag = (it.i0 - it.j0) >> 5;
    pdl_wait();  // positions come from the previous kernel

    R xi[IPT], yi[IPT], zi[IPT];
    double racc[IPT];
    f2sum facc[IPT];
    R sacc[IPT];
    V4 nxt;
    if (u_beg < u_end) nxt = mir[it.j0 + ((u_beg / S) << 5) + lane];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        // four i-atoms per thread: a 128-atom block can reach past its cluster's segment (padded to 64
        // atoms); those i-atoms are read clamped into the array and their sums are discarded
        const int iq = it.i0 + lane + 32 * q;
        const V4 p = mir[IPT == 4 ? min(iq, d.npad - 1) : iq];
        xi[q] = p.x;
        yi[q] = p.y;
        zi[q] = p.z;
        racc[q] = 0.0;
        facc[q] = {0.f, 0.f};
        sacc[q] = R(0);
    }
    V4* tile = tiles + warp * 32;
    int span = 0, tcur = -1;
    for (int u = u_beg; u < u_end; ++u) {
        const int t = u / S, k0 = (u - t * S) * L;
        const int jb = it.j0 + (t << 5);
        if (S == 1 || t != tcur) {  // stage tile t (the next one is already in flight)
            __syncwarp();
            tile[lane] = nxt;
            __syncwarp();
            if (t < t_last) nxt = mir[jb + 32 + lane];
            tcur = t;
        }
        const int valid = min(32, it.nj - (t << 5));
        const int k1 = min(k0 + L, valid);
        const bool diag = (t >= tdiag) && (t < tdiag + IPT);
        R tacc[IPT];
#pragma unroll
        for (int q = 0; q < IPT; ++q) tacc[q] = R(0);
#define SCMD_DENSITY_BODY(MASK)                                                \
    {                                                                          \
        const V4 p = tile[k];                                                  \
        _Pragma("unroll") for (int q = 0; q < IPT; ++q) {                      \
            const R dx = xi[q] - p.x, dy = yi[q] - p.y, dz = zi[q] - p.z;      \
            R r2 = fma(dx, dx, fma(dy, dy, dz * dz));                          \
            if (CUT) r2 = (r2 < rc2) ? r2 : big<R>();                          \
            if (MASK && jb + k == it.i0 + lane + 32 * q) r2 = big<R>();        \
            if (SPECIAL) {                                                     \
                const R inv = inv_r2(r2);                                      \
                tacc[q] = fma(inv * inv, inv, tacc[q]);                        \
            } else {                                                           \
                const R ir = inv_r(r2);                                        \
                tacc[q] += rpow(ir * ir, ir, mexp);                            \
            }                                                                  \
        }                                                                      \
    }
        if (!diag && k1 - k0 == L) {
#pragma unroll 8
            for (int k = k0; k < k0 + L; ++k) SCMD_DENSITY_BODY(false)
        } else {
            for (int k = k0; k < k1; ++k) SCMD_DENSITY_BODY(true)
        }
#undef SCMD_DENSITY_BODY
#pragma unroll
        for (int q = 0; q < IPT; ++q) sacc[q] += tacc[q];
        if (++span == 4 * S) {
            span = 0;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (PREC == 1)
                    facc[q] = f2_add(facc[q], (float)sacc[q]);
                else
                    racc[q] += (double)sacc[q];
                sacc[q] = R(0);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        if (PREC == 1)
            red2[warp * BI + q * 32 + lane] = f2_add(facc[q], (float)sacc[q]);
        else
            red[warp * BI + q * 32 + lane] = racc[q] + (double)sacc[q];
    }
    __syncthreads();
    cluster_wait();  // every CTA of the cluster has started: rank 0's shared memory and mbarrier are set up
    if (threadIdx.x < BI) {
        // this CTA's sum over its warps, into rank 0's inbox: rank 0 stores its own, the others push it
        // with st.async, which counts the bytes on rank 0's mbarrier
        if (PREC == 1) {
            const f2sum s2 = f2_tree_sum(red2 + threadIdx.x, W, BI);
            if (rank == 0)
                inbox2[threadIdx.x] = s2;
            else
                st_async(rank0_addr(inbox2 + rank * BI + threadIdx.x), s2, rank0_addr(&s_bar));
        } else {
            double s = 0.0;
            for (int w = 0; w < W; ++w) s += red[w * BI + threadIdx.x];
            if (rank == 0)
                inbox[threadIdx.x] = s;
            else
                st_async(rank0_addr(inbox + rank * BI + threadIdx.x), s, rank0_addr(&s_bar));
        }
    }
    if (rank != 0) return;
    if (threadIdx.x == 0) s_late = mbar_wait0(&s_bar) ? 0 : 1;
    __syncthreads();
    if (s_late) {
        if (threadIdx.x == 0) atomicOr(d.status, kStatusTimeout);
        return;
    }
    if (threadIdx.x >= BI) return;
    double tot;
    float sf = 0.f;  // MIXED: the density sum in FP32 (the high word of its double-float form)
    if (PREC == 1) {
        const f2sum t2 = f2_tree_sum(inbox2 + threadIdx.x, C, BI);
        tot = (double)t2.hi + (double)t2.lo;
        sf = t2.hi;
    } else {
        tot = 0.0;
        for (int r = 0; r < C; ++r) tot += inbox[r * BI + threadIdx.x];
    }
    const int t = threadIdx.x, i = it.i0 + t;
    const bool real = t < it.ni;
    const double rho = tot * d.pot.am;
    if (real) {
        const int q = t >> 5;  // this thread's own atom is its q-th i-atom
        V4 p;
        p.x = xi[0];
        p.y = yi[0];
        p.z = zi[0];
#pragma unroll
        for (int r = 1; r < IPT; ++r)
            if (q == r) {
                p.x = xi[r];
                p.y = yi[r];
                p.z = zi[r];
            }
        d.rho[i] = rho;
        if (PREC == 1) {
            // g = B6 rho^-1/2 = gsf sum^-1/2 on the FP32 pipe, so the FP64 work above (rho for
            // the density output) does not hold up posg; sum > 0 exactly when rho > 0
            float y = rsqrt_approx(sf);
            y = y * (1.5f - 0.5f * sf * y * y);  // one Newton step
            p.w = sf > 0.f ? d.pot.gsf * y : 0.0f;
        } else {
            p.w = rho > 0.0 ? d.pot.B6 / sqrt(rho) : 0.0;
        }
        reinterpret_cast<V4*>(d.posg)[i] = p;
    }
    if (obs) {
        double e = real ? -d.pot.eps * d.pot.c * sqrt(rho) : 0.0;
        e = warp_sum(e);
        // (a 128-atom block's groups past its cluster's padded segment belong to another item or to no one)
        if (lane == 0 && (IPT < 4 || i < d.poff[it.cl + 1])) d.part[(size_t)(i >> 5) * kObsFields + OF_EEMB] = e;
    }
}

// --------------------------------------------------------------- force pass
// Shared memory: tiles [W][32] V4 | rede [W][BI] double | inboxe [C][BI] double
//                | redf [W][BI][3] R | inboxf [C][BI][3] R
template <int PREC, int IPT, int SPECIAL, int CUT, int ENERGY>
__global__ void __launch_bounds__(512, 1) k_force(const Dev d, const Item* __restrict__ items, int C, int mode, int k_local,
                                                  int last) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    constexpr int BI = 32 * IPT;
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_bar;  // rank 0: completes when the other ranks' partials have landed
    __shared__ int s_late;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    if (rank == 0 && threadIdx.x == 0)
        mbar_setup(&s_bar, (unsigned)((C - 1) * BI * (3 * sizeof(typename Tr<PREC>::R) + (ENERGY ? 8 : 0))));
    cluster_arrive_relaxed();
    pdl_launch_dependents();
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Item it = load_item<BI>(d, items, C);
    V4* tiles = reinterpret_cast<V4*>(smem);
    double* rede = reinterpret_cast<double*>(smem + (size_t)W * 32 * sizeof(V4));
    double* inboxe = rede + W * BI;
    R* redf = reinterpret_cast<R*>(inboxe + C * BI);
    R* inboxf = redf + W * BI * 3;
    const V4* pg = reinterpret_cast<const V4*>(d.posg);
    const R A = PREC == 1 ? (R)d.pot.A9f : (R)d.pot.A9;  // no FP64 conversion in MIXED
    const R rc2 = PREC == 1 ? (R)d.pot.rcut2f : (R)d.pot.rcut2;
    const int nexp = d.pot.n, mexp = d.pot.m;
    constexpr int S = SplitOf<PREC>::S, L = 32 / S;
    const int ntile = (it.nj + 31) >> 5, nunit = ntile * S;
    const int Q = C * W, qi = rank * W + warp;
    const int u_beg = (int)(((long long)nunit * qi) / Q), u_end = (int)(((long long)nunit * (qi + 1)) / Q);
    const int t_last = (u_end - 1) / S;
    const int tdiag = (it.i0 - it.j0) >> 5;
    // epilogue owner: rank 0, thread t < BI owns atom i0 + t
    const bool owner = rank == 0 && threadIdx.x < BI;
    const bool oreal = owner && (int)threadIdx.x < it.ni;
    const int io = it.i0 + threadIdx.x;
    const Run* __restrict__ run = d.run;
    const bool integrate = mode == 2;
    pdl_wait();  // posg comes from the density pass; x, v and the noise from earlier kernels
    // The epilogue's inputs are copied into this owner's shared-memory slot with cp.async
    // before the pair loop (no register, no stall) and waited for only after it.
    const uintptr_t slot0 = (reinterpret_cast<uintptr_t>(inboxf + C * BI * 3) + 15) & ~uintptr_t(15);
    EpiSlot* slot = reinterpret_cast<EpiSlot*>(slot0) + (owner ? threadIdx.x : 0);
    if (integrate && oreal) {
        const int np = d.npad;
        cp_async8(&slot->v[0], d.v + io);
        cp_async8(&slot->v[1], d.v + np + io);
        cp_async8(&slot->v[2], d.v + 2 * np + io);
        cp_async8(&slot->x[0], d.x + io);
        cp_async8(&slot->x[1], d.x + np + io);
        cp_async8(&slot->x[2], d.x + 2 * np + io);
        cp_async8(&slot->hs, d.hs + io);
        cp_async8(&slot->m, d.mass + io);
        if (PREC == 1) {
            cp_async8(&slot->o[0], d.origin + 3 * it.cl);
            cp_async8(&slot->o[1], d.origin + 3 * it.cl + 1);
            cp_async8(&slot->o[2], d.origin + 3 * it.cl + 2);
            if (!last) {
                cp_async16(&slot->nz, d.noise + (size_t)(k_local + 1) * np + io);  // step base + k_local + 1
                cp_async4(&slot->sig0, d.sig0 + io);
            }
        }
        cp_async_commit();
    }

    R xi[IPT], yi[IPT], zi[IPT], gi[IPT];
    R fx[IPT], fy[IPT], fz[IPT], sx[IPT], sy[IPT], sz[IPT];
    R es[IPT];
    double ea[IPT];
    V4 nxt;
    if (u_beg < u_end) nxt = pg[it.j0 + ((u_beg / S) << 5) + lane];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const V4 p = pg[it.i0 + lane + 32 * q];
        xi[q] = p.x;
        yi[q] = p.y;
        zi[q] = p.z;
        gi[q] = p.w;
        fx[q] = fy[q] = fz[q] = R(0);
        sx[q] = sy[q] = sz[q] = R(0);
        es[q] = R(0);
        ea[q] = 0.0;
    }
    V4* tile = tiles + warp * 32;
    int span = 0, tcur = -1;
    for (int u = u_beg; u < u_end; ++u) {
        const int t = u / S, k0 = (u - t * S) * L;
        const int jb = it.j0 + (t << 5);
        if (S == 1 || t != tcur) {
            __syncwarp();
            tile[lane] = nxt;
            __syncwarp();
            if (t < t_last) nxt = pg[jb + 32 + lane];
            tcur = t;
        }
        const int valid = min(32, it.nj - (t << 5));
        const int k1 = min(k0 + L, valid);
        const bool diag = (t >= tdiag) && (t < tdiag + IPT);
        R tx[IPT], ty[IPT], tz[IPT], te[IPT];
#pragma unroll
        for (int q = 0; q < IPT; ++q) tx[q] = ty[q] = tz[q] = te[q] = R(0);
#define SCMD_FORCE_BODY(MASK)                                                  \
    {                                                                          \
        const V4 p = tile[k];                                                  \
        _Pragma("unroll") for (int q = 0; q < IPT; ++q) {                      \
            const R dx = xi[q] - p.x, dy = yi[q] - p.y, dz = zi[q] - p.z;      \
            R r2 = fma(dx, dx, fma(dy, dy, dz * dz));                          \
            if (CUT) r2 = (r2 < rc2) ? r2 : big<R>();                          \
            if (MASK && jb + k == it.i0 + lane + 32 * q) r2 = big<R>();        \
            const R ir = inv_r(r2);                                            \
            const R inv = ir * ir;                                             \
            R coef, rn;                                                        \
            if (SPECIAL) {                                                     \
                const R inv2 = inv * inv, inv4 = inv2 * inv2;                  \
                coef = inv4 * fma(A, inv * ir, -(gi[q] + p.w));                \
                rn = inv4 * ir;                                                \
            } else {                                                           \
                rn = rpow(inv, ir, nexp);                                      \
                const R rm = rpow(inv, ir, mexp);                              \
                coef = inv * (A * rn - (gi[q] + p.w) * rm);                    \
            }                                                                  \
            tx[q] = fma(coef, dx, tx[q]);                                      \
            ty[q] = fma(coef, dy, ty[q]);                                      \
            tz[q] = fma(coef, dz, tz[q]);                                      \
            if (ENERGY) te[q] += rn;                                           \
        }                                                                      \
    }
        if (!diag && k1 - k0 == L) {
#pragma unroll 8
            for (int k = k0; k < k0 + L; ++k) SCMD_FORCE_BODY(false)
        } else {
            for (int k = k0; k < k1; ++k) SCMD_FORCE_BODY(true)
        }
#undef SCMD_FORCE_BODY
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            sx[q] += tx[q];
            sy[q] += ty[q];
            sz[q] += tz[q];
            if (ENERGY) es[q] += te[q];
        }
        if (++span == 4 * S) {
            span = 0;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                fx[q] += sx[q];
                fy[q] += sy[q];
                fz[q] += sz[q];
                sx[q] = sy[q] = sz[q] = R(0);
                if (ENERGY) {
                    ea[q] += (double)es[q];
                    es[q] = R(0);
                }
            }
        }
    }
    // MIXED steps that go on to the next step: the step coefficients for the split epilogue
    // below, loaded here so that their latency hides behind the reductions.
    constexpr bool kSplit = PREC == 1 && IPT == 1;
    int kind0 = 2;
    double c_h = 0.0, c_hk = 0.0, c_c1 = 0.0, c_dt = 0.0;
    if (kSplit && integrate && !last && rank == 0) {
        kind0 = run->kind;
        c_h = run->h;
        c_hk = run->hk;
        c_c1 = run->c1;
        c_dt = run->dt;
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int sidx = warp * BI + q * 32 + lane;
        redf[3 * sidx + 0] = fx[q] + sx[q];
        redf[3 * sidx + 1] = fy[q] + sy[q];
        redf[3 * sidx + 2] = fz[q] + sz[q];
        if (ENERGY) rede[sidx] = ea[q] + (double)es[q];
    }
    __syncthreads();
    cluster_wait();  // every CTA of the cluster has started
    if (threadIdx.x < BI) {
        R ax = R(0), ay = R(0), az = R(0);
        double ae = 0.0;
        for (int w = 0; w < W; ++w) {
            const int sidx = w * BI + threadIdx.x;
            ax += redf[3 * sidx];
            ay += redf[3 * sidx + 1];
            az += redf[3 * sidx + 2];
            if (ENERGY) ae += rede[sidx];
        }
        R* dst = inboxf + 3 * (rank * BI + threadIdx.x);
        if (rank == 0) {
            dst[0] = ax;
            dst[1] = ay;
            dst[2] = az;
            if (ENERGY) inboxe[threadIdx.x] = ae;
        } else {  // pushed into rank 0's inbox; the bytes count on rank 0's mbarrier
            const unsigned bar = rank0_addr(&s_bar);
            st_async(rank0_addr(dst), ax, bar);
            st_async(rank0_addr(dst + 1), ay, bar);
            st_async(rank0_addr(dst + 2), az, bar);
            if (ENERGY) st_async(rank0_addr(inboxe + rank * BI + threadIdx.x), ae, bar);
        }
    }
    if (rank != 0) return;
    if (threadIdx.x == 0) s_late = mbar_wait0(&s_bar) ? 0 : 1;
    __syncthreads();
    if (s_late) {
        if (threadIdx.x == 0) atomicOr(d.status, kStatusTimeout);
        return;
    }
    // Split epilogue (MIXED, NVE or Langevin, not the chunk's last step). FP64 runs at 1/64 of
    // the FP32 rate here and a warp instruction holds its sub-partition's FP64 unit for ~68
    // cycles, so one warp integrating all three components of its 32 atoms is ~27 FP64
    // instructions in a row at the end of the pass. The components are independent, so each of
    // up to 3 * IPT warps (on different sub-partitions) takes one component of 32 atoms, with
    // the same operations in the same order as the one-warp form below. This pays where a
    // launch is one short wave (small clusters, IPT = 1). The IPT = 2 shapes serve large N,
    // where many CTAs share each SM and the epilogue hides behind other CTAs' pair loops; there
    // the split measured slower (its extra loads and barrier), so it is compiled in for IPT = 1.
    constexpr int NT = 3 * IPT;
    const int NW = W < NT ? W : NT;
    const bool split = kSplit && integrate && !last && kind0 != 2;
    if (!owner && !(split && rank == 0 && warp < NW)) return;
    R Fx = R(0), Fy = R(0), Fz = R(0);
    double Ep = 0.0;
    const int i = io, np = d.npad;
    const bool real = oreal;
    const int group = i >> 5;
    if (owner) {
        for (int r = 0; r < C; ++r) {
            const R* rf = inboxf + 3 * (r * BI + threadIdx.x);
            Fx += rf[0];
            Fy += rf[1];
            Fz += rf[2];
            if (ENERGY) Ep += inboxe[r * BI + threadIdx.x];
        }
        R* fo = reinterpret_cast<R*>(d.f);
        if (real) {
            fo[i] = Fx;
            fo[np + i] = Fy;
            fo[2 * np + i] = Fz;
            if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(d.status, 1);
        }
    }
    if (split) {
        R* fsh = redf;  // free again after the cluster barrier: F by component, [3][BI]
        const EpiSlot* slots = reinterpret_cast<const EpiSlot*>(slot0);
        if (owner) {
            fsh[threadIdx.x] = Fx;
            fsh[BI + threadIdx.x] = Fy;
            fsh[2 * BI + threadIdx.x] = Fz;
            cp_async_wait_all();
            if (ENERGY) {  // observables are due at step + 1: the owner warp sums them as below
                const double hs = slot->hs, m = real ? slot->m : 0.0;
                const double vx = fma(hs, (double)Fx, slot->v[0]), vy = fma(hs, (double)Fy, slot->v[1]),
                             vz = fma(hs, (double)Fz, slot->v[2]);
                const double e = warp_sum(real ? Ep : 0.0);
                if (lane == 0) d.part[(size_t)group * kObsFields + OF_EPAIR] = e;
                obs_position_partials(d, group, real, m, slot->x[0], slot->x[1], slot->x[2], lane);
                obs_velocity_partials(d, group, real, m, slot->x[0], slot->x[1], slot->x[2], vx, vy, vz, lane);
            }
        }
        bar_sync_first(NW * 32);  // F and every owner's epilogue slot are in shared memory
        float* mirf = reinterpret_cast<float*>(d.mirror);
        for (int task = warp; task < NT; task += NW) {
            const int c = task / IPT, t = (task - c * IPT) * 32 + lane;
            if (t >= it.ni) continue;
            const int ia = it.i0 + t;
            const EpiSlot* s = slots + t;
            const double F = (double)fsh[c * BI + t];
            const double hs = s->hs;
            const double vv = fma(hs, F, s->v[c]);  // end of this step (second half kick)
            double u = fma(hs, F, vv);              // next step: first half kick
            double x;
            if (kind0 == 1) {  // A O A
                const double nzc = (double)(s->sig0 * reinterpret_cast<const float*>(&s->nz)[c]);
                x = fma(c_hk, u, fma(c_h, nzc, s->x[c]));
                u = fma(c_c1, u, nzc);
            } else {  // A A
                x = fma(c_dt, u, s->x[c]);
            }
            mirf[4 * ia + c] = (float)(x - s->o[c]);  // the .w of the mirror stays 0
            d.v[c * np + ia] = u;
            d.x[c * np + ia] = x;
            if (!(finite_bits(x) && finite_bits(u))) atomicOr(d.status, 1);
        }
        return;
    }
    if (mode == 1) {
        // fresh evaluation: all observable partials at the current (x, v)
        const double mm = real ? d.mass[i] : 0.0;
        if (ENERGY) {
            const double e = warp_sum(real ? Ep : 0.0);
            if (lane == 0) d.part[(size_t)group * kObsFields + OF_EPAIR] = e;
        }
        const double x = real ? d.x[i] : 0.0, y = real ? d.x[np + i] : 0.0, z = real ? d.x[2 * np + i] : 0.0;
        const double vx = real ? d.v[i] : 0.0, vy = real ? d.v[np + i] : 0.0, vz = real ? d.v[2 * np + i] : 0.0;
        obs_velocity_partials(d, group, real, mm, x, y, z, vx, vy, vz, lane);
        obs_position_partials(d, group, real, mm, x, y, z, lane);
    } else if (mode == 2) {
        const Run* rr = run;
        const int r_kind = rr->kind;
        cp_async_wait_all();
        const double vx0 = slot->v[0], vy0 = slot->v[1], vz0 = slot->v[2];
        const double xx0 = slot->x[0], yy0 = slot->x[1], zz0 = slot->x[2];
        const double hs = slot->hs, m = real ? slot->m : 0.0;
        const double Fxd = (double)Fx, Fyd = (double)Fy, Fzd = (double)Fz;
        // velocities at the end of this step (second half kick)
        const double vx = fma(hs, Fxd, vx0), vy = fma(hs, Fyd, vy0), vz = fma(hs, Fzd, vz0);
        if (ENERGY) {  // observables are due at step + 1 (the host compiles ENERGY in only then)
            const double e = warp_sum(real ? Ep : 0.0);
            if (lane == 0) d.part[(size_t)group * kObsFields + OF_EPAIR] = e;
            obs_position_partials(d, group, real, m, xx0, yy0, zz0, lane);
            if (r_kind != 2) obs_velocity_partials(d, group, real, m, xx0, yy0, zz0, vx, vy, vz, lane);
        }
        if (r_kind == 2) {
            if (real) {
                d.v[i] = vx;
                d.v[np + i] = vy;
                d.v[2 * np + i] = vz;
            }
            const double ke2 = warp_sum(real ? m * (vx * vx + vy * vy + vz * vz) : 0.0);
            if (lane == 0) d.ke_grp[group] = ke2;
        } else if (real) {
            if (last) {
                d.v[i] = vx;
                d.v[np + i] = vy;
                d.v[2 * np + i] = vz;
            } else {
                // next step (same arithmetic as begin_step): first half kick, then A O A or A A
                double ux = fma(hs, Fxd, vx), uy = fma(hs, Fyd, vy), uz = fma(hs, Fzd, vz);
                double x, y, z;
                if (r_kind == 1) {
                    const double h = rr->h, hk = rr->hk, c1 = rr->c1;
                    double nx, ny, nz;
                    if (PREC == 1) {
                        const float sg = slot->sig0;
                        const float4 w = slot->nz;
                        nx = (double)(sg * w.x);
                        ny = (double)(sg * w.y);
                        nz = (double)(sg * w.z);
                    } else {
                        const Run r = *rr;
                        const int64_t s1 = *d.step_base + k_local + 1;
                        double w[3];
                        normals_f64(r.seed, (uint32_t)it.cl, s1, (uint32_t)(i - it.j0), w);
                        const double sig = sqrt(r.noise_k * fmax(ramp_T(r, s1), 0.0) / m);
                        nx = sig * w[0];
                        ny = sig * w[1];
                        nz = sig * w[2];
                    }
                    x = fma(hk, ux, fma(h, nx, xx0));
                    y = fma(hk, uy, fma(h, ny, yy0));
                    z = fma(hk, uz, fma(h, nz, zz0));
                    ux = fma(c1, ux, nx);
                    uy = fma(c1, uy, ny);
                    uz = fma(c1, uz, nz);
                } else {
                    const double dt = rr->dt;
                    x = fma(dt, ux, xx0);
                    y = fma(dt, uy, yy0);
                    z = fma(dt, uz, zz0);
                }
                if (PREC == 1) {
                    float4 p;
                    p.x = (float)(x - slot->o[0]);
                    p.y = (float)(y - slot->o[1]);
                    p.z = (float)(z - slot->o[2]);
                    p.w = 0.f;
                    reinterpret_cast<float4*>(d.mirror)[i] = p;
                } else {
                    store_mirror<PREC>(d, i, it.cl, x, y, z);
                }
                d.v[i] = ux;
                d.v[np + i] = uy;
                d.v[2 * np + i] = uz;
                d.x[i] = x;
                d.x[np + i] = y;
                d.x[2 * np + i] = z;
                if (!(finite_bits(x) && finite_bits(y) && finite_bits(z) && finite_bits(ux) && finite_bits(uy) &&
                      finite_bits(uz)))
                    atomicOr(d.status, 1);
            }
        }
    }
}

// ------------------------------------------------------------ per-atom kernels
// One 32-thread CTA per 32-atom group; the group's cluster comes from a table.
template <int PREC> __global__ void k_start(const Dev d, int k_local) {
    pdl_launch_dependents();
    pdl_wait();
    const int g = blockIdx.x, lane = threadIdx.x, i = g * 32 + lane;
    const int cl = d.cl_of_group[g];
    const int a = i - d.poff[cl];
    if (a >= d.nreal[cl]) return;
    const Run r = *d.run;
    double fx, fy, fz;
    load_force<PREC>(d, i, fx, fy, fz);
    begin_step<PREC>(d, r, i, cl, a, *d.step_base + k_local, fx, fy, fz, k_local);
}

template <int PREC> __global__ void k_berendsen(const Dev d, int k_local, int last) {
    pdl_launch_dependents();
    pdl_wait();
    const int g = blockIdx.x, lane = threadIdx.x, i = g * 32 + lane;
    const int cl = d.cl_of_group[g];
    const int g0 = d.poff[cl] >> 5, g1 = d.poff[cl + 1] >> 5;
    double ke2 = 0.0;
    for (int k = g0 + lane; k < g1; k += 32) ke2 += d.ke_grp[k];
    ke2 = warp_sum(ke2);
    const Run r = *d.run;
    const int64_t step = *d.step_base + k_local;  // completed step -> step + 1
    const int n = d.nreal[cl];
    const double T_inst = ke2 / (d.conv * 3.0 * n * r.kb);
    const double Tt = ramp_T(r, step);
    const double lam = T_inst > 0.0 ? sqrt(1.0 + r.dt_over_tau * (Tt / T_inst - 1.0)) : 1.0;
    const int a = i - d.poff[cl];
    const bool real = a < n;
    const int np = d.npad;
    double vx = 0.0, vy = 0.0, vz = 0.0, m = 0.0;
    if (real) {
        m = d.mass[i];
        vx = d.v[i] * lam;
        vy = d.v[np + i] * lam;
        vz = d.v[2 * np + i] * lam;
        d.v[i] = vx;
        d.v[np + i] = vy;
        d.v[2 * np + i] = vz;
    }
    const int64_t next = step + 1;
    if (r.obs_every > 0 && next % r.obs_every == 0) {
        const double x = real ? d.x[i] : 0.0, y = real ? d.x[np + i] : 0.0, z = real ? d.x[2 * np + i] : 0.0;
        obs_velocity_partials(d, g, real, m, x, y, z, vx, vy, vz, lane);
    }
    if (!last && real) {
        double fx, fy, fz;
        load_force<PREC>(d, i, fx, fy, fz);
        begin_step<PREC>(d, r, i, cl, a, next, fx, fy, fz, -1);
    }
}

// Mirror of the current positions relative to the cluster origins.
template <int PREC> __global__ void k_mirror(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int g = blockIdx.x, lane = threadIdx.x, i = g * 32 + lane;
    const int cl = d.cl_of_group[g];
    if (i - d.poff[cl] >= d.nreal[cl]) return;
    store_mirror<PREC>(d, i, cl, d.x[i], d.x[d.npad + i], d.x[2 * d.npad + i]);
}

// Mirror origin of each cluster = its centre of mass (one CTA of 32 threads per cluster).
__global__ void k_origin(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int cl = blockIdx.x, lane = threadIdx.x;
    const int b = d.poff[cl], n = d.nreal[cl], np = d.npad;
    double sx = 0.0, sy = 0.0, sz = 0.0, sm = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double m = d.mass[b + k];
        sx += m * d.x[b + k];
        sy += m * d.x[np + b + k];
        sz += m * d.x[2 * np + b + k];
        sm += m;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    sz = warp_sum(sz);
    sm = warp_sum(sm);
    if (lane == 0) {
        d.origin[3 * cl] = sm > 0.0 ? sx / sm : 0.0;
        d.origin[3 * cl + 1] = sm > 0.0 ? sy / sm : 0.0;
        d.origin[3 * cl + 2] = sm > 0.0 ? sz / sm : 0.0;
    }
}

// Observables of every cluster from the group partials (one CTA of 32 threads per cluster).
// slot_mode 0: the "current" slot (index hist_cap); 1: ring slot of step base + k_local + 1.
__global__ void k_obs_reduce(const Dev d, int k_local, int slot_mode) {
    pdl_launch_dependents();
    pdl_wait();
    const int cl = blockIdx.x, lane = threadIdx.x;
    const int g0 = d.poff[cl] >> 5, g1 = d.poff[cl + 1] >> 5;
    double s[kObsFields];
#pragma unroll
    for (int f = 0; f < kObsFields; ++f) s[f] = 0.0;
    for (int g = g0 + lane; g < g1; g += 32) {
        const double* p = d.part + (size_t)g * kObsFields;
#pragma unroll
        for (int f = 0; f < 13; ++f) s[f] += p[f];
    }
#pragma unroll
    for (int f = 0; f < 13; ++f) s[f] = warp_sum(s[f]);
    if (lane != 0) return;
    const Run r = *d.run;
    const int64_t step = *d.step_base + k_local + (slot_mode ? 1 : 0);
    const int slot = slot_mode ? (int)((step / r.obs_every) % r.hist_cap) : r.hist_cap;
    double* h = d.hist + ((size_t)slot * d.B + cl) * kHistFields;
    const int n = d.nreal[cl];
    const double epot = s[OF_EEMB] + d.pot.ecoef * s[OF_EPAIR];
    const double ekin = 0.5 * s[OF_KE2] / d.conv;
    const double M = s[OF_MASS];
    double com[3];
    for (int k = 0; k < 3; ++k) com[k] = M > 0.0 ? s[OF_MX + k] / M : 0.0;
    const double* P = s + OF_P;
    h[0] = epot;
    h[1] = ekin;
    h[2] = epot + ekin;
    h[3] = n > 0 ? 2.0 * ekin / (3.0 * n * r.kb) : 0.0;
    h[4] = com[0];
    h[5] = com[1];
    h[6] = com[2];
    h[7] = P[0];
    h[8] = P[1];
    h[9] = P[2];
    h[10] = s[OF_L] - (com[1] * P[2] - com[2] * P[1]);
    h[11] = s[OF_L + 1] - (com[2] * P[0] - com[0] * P[2]);
    h[12] = s[OF_L + 2] - (com[0] * P[1] - com[1] * P[0]);
    h[13] = (double)step;
    h[14] = 0.0;  // time is filled in by the host from the step
    const bool bad = !isfinite(h[2]) || ((*d.status) & 1);
    h[15] = bad ? 1.0 : 0.0;
}

__global__ void k_advance(const Dev d, int n) {
    pdl_launch_dependents();
    pdl_wait();
    *d.step_base += n;
}

// Langevin normals of steps base .. base + M - 1 for every atom, ahead of the chunk
// (MIXED): noise[m][i] = the three FP32 Box-Muller normals of step base + m, times
// sqrt(T) of that step's target temperature (the per-atom factor sig0 is applied later).
__global__ void k_noise(const Dev d, int M) {
    pdl_launch_dependents();
    pdl_wait();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)M * d.npad) return;
    const int m = (int)(idx / d.npad), i = (int)(idx - (long long)m * d.npad);
    const int cl = d.cl_of_group[i >> 5];
    const int a = i - d.poff[cl];
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a < d.nreal[cl]) {
        const Run& r = *d.run;
        float zz[3];
        const int64_t step = *d.step_base + m;
        normals_f32(r.seed, (uint32_t)cl, step, (uint32_t)a, zz);
        const float sT = sqrtf((float)fmax(ramp_T(r, step), 0.0));
        out = make_float4(zz[0] * sT, zz[1] * sT, zz[2] * sT, 0.f);
    }
    d.noise[idx] = out;
}

// Per-atom factors of the current md_step call: h conv / m and sqrt((1 - c1^2) k_B conv / m).
__global__ void k_prepare(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.npad) return;
    const Run r = *d.run;
    const double m = d.mass[i];
    const_cast<double*>(d.hs)[i] = r.h * d.conv / m;
    const_cast<float*>(d.sig0)[i] = (float)sqrt(r.noise_k / m);
}

__global__ void k_philox(const uint32_t* in, uint32_t* out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t c[4] = {in[6 * k], in[6 * k + 1], in[6 * k + 2], in[6 * k + 3]};
    philox4x32_10(c, in[6 * k + 4], in[6 * k + 5]);
    for (int w = 0; w < 4; ++w) out[4 * k + w] = c[w];
}

__global__ void k_normals(uint64_t seed, uint32_t cl, int64_t step, int n, int prec, double* out) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    if (prec == 1) {
        float z[3];
        normals_f32(seed, cl, step, (uint32_t)a, z);
        for (int c = 0; c < 3; ++c) out[3 * a + c] = (double)z[c];
    } else {
        double z[3];
        normals_f64(seed, cl, step, (uint32_t)a, z);
        for (int c = 0; c < 3; ++c) out[3 * a + c] = z[c];
    }
}

// ---------------------------------------------------------------- launchers
size_t pass_smem_bytes(int prec, Shape sh, int which) {
    const size_t v4 = prec == 1 ? sizeof(float4) : sizeof(dbl4);
    const size_t r = prec == 1 ? sizeof(float) : sizeof(double);
    const size_t BI = 32 * (size_t)sh.ipt, W = sh.warps, C = sh.cluster;
    const size_t tiles = W * 32 * v4;
    const size_t dens = (W + C) * BI * sizeof(double);
    if (which == 0) return tiles + dens;  // density pass: tiles, per-warp partials, the cluster inbox
    const size_t force = (W + C) * BI * sizeof(double) + (W + C) * BI * 3 * r;
    // force pass: the epilogue slots follow the reduction buffers, 16-byte aligned
    const size_t force_slots = ((tiles + force + 15) / 16) * 16 - tiles + BI * sizeof(EpiSlot);
    return tiles + (dens > force_slots ? dens : force_slots);
}

template <int PREC, int IPT, int SPECIAL, int CUT>
static cudaError_t density_t(const Dev& d, const Item* items, int nitems, Shape sh, int obs, cudaStream_t s) {
    return launch_cluster(k_density<PREC, IPT, SPECIAL, CUT>, nitems * sh.cluster, sh.warps * 32,
                          pass_smem_bytes(PREC, sh, 0), sh.cluster, s, d, items, sh.cluster, obs);
}
template <int PREC, int IPT, int SPECIAL, int CUT, int ENERGY>
static cudaError_t force_t(const Dev& d, const Item* items, int nitems, Shape sh, int mode, int k_local, int last,
                           cudaStream_t s) {
    return launch_cluster(k_force<PREC, IPT, SPECIAL, CUT, ENERGY>, nitems * sh.cluster, sh.warps * 32,
                          pass_smem_bytes(PREC, sh, 1), sh.cluster, s, d, items, sh.cluster, mode, k_local, last);
}

template <int PREC, int IPT>
static cudaError_t density_p(const Dev& d, const Item* it, int n, Shape sh, int obs, cudaStream_t s) {
    const bool sp = d.pot.special != 0, cut = d.pot.rcut > 0.0;
    if (sp && !cut) return density_t<PREC, IPT, 1, 0>(d, it, n, sh, obs, s);
    if (sp && cut) return density_t<PREC, IPT, 1, 1>(d, it, n, sh, obs, s);
    if (!sp && !cut) return density_t<PREC, IPT, 0, 0>(d, it, n, sh, obs, s);
    return density_t<PREC, IPT, 0, 1>(d, it, n, sh, obs, s);
}
template <int PREC, int IPT, int ENERGY>
static cudaError_t force_p(const Dev& d, const Item* it, int n, Shape sh, int mode, int k, int last, cudaStream_t s) {
    const bool sp = d.pot.special != 0, cut = d.pot.rcut > 0.0;
    if (sp && !cut) return force_t<PREC, IPT, 1, 0, ENERGY>(d, it, n, sh, mode, k, last, s);
    if (sp && cut) return force_t<PREC, IPT, 1, 1, ENERGY>(d, it, n, sh, mode, k, last, s);
    if (!sp && !cut) return force_t<PREC, IPT, 0, 0, ENERGY>(d, it, n, sh, mode, k, last, s);
    return force_t<PREC, IPT, 0, 1, ENERGY>(d, it, n, sh, mode, k, last, s);
}

cudaError_t launch_density(const Dev& d, const Item* items, int nitems, Shape sh, int obs, cudaStream_t s) {
    if (d.h_nunits > 0) return launch_h_density(d, obs, s);  // FP64, each pair once
    if (nitems <= 0) return cudaSuccess;
    if (d.prec == 1) {
        if (sh.ipt == 4) return density_p<1, 4>(d, items, nitems, sh, obs, s);
        return sh.ipt == 2 ? density_p<1, 2>(d, items, nitems, sh, obs, s) : density_p<1, 1>(d, items, nitems, sh, obs, s);
    }
    if (sh.ipt == 4) return density_p<0, 4>(d, items, nitems, sh, obs, s);
    return sh.ipt == 2 ? density_p<0, 2>(d, items, nitems, sh, obs, s) : density_p<0, 1>(d, items, nitems, sh, obs, s);
}

cudaError_t launch_force(const Dev& d, const Item* items, int nitems, Shape sh, int mode, int k_local, int flags,
                         cudaStream_t s) {
    if (d.h_nunits > 0) return launch_h_force(d, mode, k_local, flags, s);  // FP64, each pair once
    if (nitems <= 0) return cudaSuccess;
    // ENERGY (pair-energy accumulation in the inner loop) is compiled in for fresh
    // evaluations (mode 1) and for MD steps whose end is an observation (flag bit 1).
    const bool energy = (mode == 1) || (mode == 2 && (flags & 2));
    const int lst = flags & 1;
    if (d.prec == 1) {
        if (sh.ipt == 2)
            return energy ? force_p<1, 2, 1>(d, items, nitems, sh, mode, k_local, lst, s)
                          : force_p<1, 2, 0>(d, items, nitems, sh, mode, k_local, lst, s);
        return energy ? force_p<1, 1, 1>(d, items, nitems, sh, mode, k_local, lst, s)
                      : force_p<1, 1, 0>(d, items, nitems, sh, mode, k_local, lst, s);
    }
    if (sh.ipt == 2)
        return energy ? force_p<0, 2, 1>(d, items, nitems, sh, mode, k_local, lst, s)
                      : force_p<0, 2, 0>(d, items, nitems, sh, mode, k_local, lst, s);
    return energy ? force_p<0, 1, 1>(d, items, nitems, sh, mode, k_local, lst, s)
                  : force_p<0, 1, 0>(d, items, nitems, sh, mode, k_local, lst, s);
}

cudaError_t launch_start(const Dev& d, int k_local, cudaStream_t s) {
    if (d.prec == 1)
        return launch_ex(k_start<1>, d.ngroups, 32, 0, 0, s, d, k_local);
    return launch_ex(k_start<0>, d.ngroups, 32, 0, 0, s, d, k_local);
}
cudaError_t launch_berendsen(const Dev& d, int k_local, int last, cudaStream_t s) {
    if (d.prec == 1)
        return launch_ex(k_berendsen<1>, d.ngroups, 32, 0, 0, s, d, k_local, last);
    return launch_ex(k_berendsen<0>, d.ngroups, 32, 0, 0, s, d, k_local, last);
}
cudaError_t launch_mirror(const Dev& d, cudaStream_t s) {
    if (d.prec == 1)
        return launch_ex(k_mirror<1>, d.ngroups, 32, 0, 0, s, d);
    return launch_ex(k_mirror<0>, d.ngroups, 32, 0, 0, s, d);
}
cudaError_t launch_origin(const Dev& d, cudaStream_t s) {
    return launch_ex(k_origin, d.B, 32, 0, 0, s, d);
}
cudaError_t launch_noise(const Dev& d, int M, cudaStream_t s) {
    const long long n = (long long)M * d.npad;
    return launch_ex(k_noise, (int)((n + 255) / 256), 256, 0, 0, s, d, M);
}
cudaError_t launch_prepare(const Dev& d, cudaStream_t s) {
    return launch_ex(k_prepare, (d.npad + 255) / 256, 256, 0, 0, s, d);
}
cudaError_t launch_obs_reduce(const Dev& d, int k_local, int slot_mode, cudaStream_t s) {
    return launch_ex(k_obs_reduce, d.B, 32, 0, 0, s, d, k_local, slot_mode);
}
cudaError_t launch_advance(const Dev& d, int n, cudaStream_t s) {
    return launch_ex(k_advance, 1, 1, 0, 0, s, d, n);
}
cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_philox<<<(n + 127) / 128, 128, 0, s>>>(in, out, n);
    return cudaGetLastError();
}
cudaError_t launch_normals(uint64_t seed, uint32_t cl, int64_t step, int n, int prec, double* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_normals<<<(n + 127) / 128, 128, 0, s>>>(seed, cl, step, n, prec, out);
    return cudaGetLastError();
}

template <class K> static cudaError_t allow_smem(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}
template <int PREC, int IPT, int SP, int CUT> static cudaError_t cfg_one() {
    cudaError_t e = allow_smem(k_density<PREC, IPT, SP, CUT>);
    if (e == cudaSuccess) e = allow_smem(k_force<PREC, IPT, SP, CUT, 0>);
    if (e == cudaSuccess) e = allow_smem(k_force<PREC, IPT, SP, CUT, 1>);
    return e;
}
template <int PREC, int IPT> static cudaError_t cfg_ipt() {
    cudaError_t e = cfg_one<PREC, IPT, 1, 0>();
    if (e == cudaSuccess) e = cfg_one<PREC, IPT, 1, 1>();
    if (e == cudaSuccess) e = cfg_one<PREC, IPT, 0, 0>();
    if (e == cudaSuccess) e = cfg_one<PREC, IPT, 0, 1>();
    return e;
}
template <int PREC> static cudaError_t cfg_density4() {
    cudaError_t e = allow_smem(k_density<PREC, 4, 1, 0>);
    if (e == cudaSuccess) e = allow_smem(k_density<PREC, 4, 1, 1>);
    if (e == cudaSuccess) e = allow_smem(k_density<PREC, 4, 0, 0>);
    if (e == cudaSuccess) e = allow_smem(k_density<PREC, 4, 0, 1>);
    return e;
}
cudaError_t configure_kernels() {
    cudaError_t e = cfg_ipt<1, 1>();
    if (e == cudaSuccess) e = cfg_ipt<1, 2>();
    if (e == cudaSuccess) e = cfg_ipt<0, 1>();
    if (e == cudaSuccess) e = cfg_ipt<0, 2>();
    if (e == cudaSuccess) e = cfg_density4<1>();
    if (e == cudaSuccess) e = cfg_density4<0>();
    return e;
}

}  // namespace scmd
