// scmd_cells.cu -- the cell-list path of the two pair passes (strict cutoff r < rcut).
//
// The paper evaluates every pair and names efficient cutoff schemes as work in progress
// (Sec. II). With rcut > 0 a context may instead give each cluster a cubic grid of G^3 cells of
// side h > rcut, fixed when the context is created: the cube [-E, E)^3 around the cluster's
// origin (the centre of mass that the MIXED pair coordinates are measured from), with E a
// margin beyond the cluster's radius. Atoms outside the cube are clamped into its border
// cells; clamping is monotone per axis and moves an atom only outward, so two atoms closer than
// rcut are still found by the stencil below. Per MD step:
//   k_cell_clear, k_cell_bin : atoms binned into cells of fixed capacity (atomic slots;
//                              an overflow sets status bit 1, reported by the host);
//   k_cell_sort              : each cell's list sorted by (octant, atom index), so the order of
//                              every sum below and hence the results are independent of the order
//                              in which the atomic slots were taken;
//   k_cell_density           : rho_i over the neighbour octants (Eq. 2 with the cutoff);
//   k_cell_force             : F_i over the neighbour octants (-grad of Eq. 1 with the cutoff),
//                              then the integrator step of the all-pairs path.
// Octants: each cell is split into 2 x 2 x 2 octants of side h/2 > rcut/2. Two atoms closer than
// rcut lie at most two octants apart per axis, so the atoms of one home octant need only the
// 5 x 5 x 5 octants around it: 125 of the 216 octants of the 27 cells around the home cell, which
// cuts the pairs tested by ~42 % against whole cells.
// Pair coordinates are relative to cell centres: when the atoms are binned, each cell stores its
// atoms' offsets x - centre (rounded once from the FP64 state to the pass precision), and a CTA
// moves a neighbour cell's offsets to its own centre by adding (k - l) h, which is exact in FP32
// (h is a binary32 value). In MIXED mode a coordinate is then off by at most about
// ulp(1.5 h) ~ 5e-7 A whatever the cluster's size, where offsets from one origin per cluster
// would carry ulp(R) (about 2e-6 A at R = 50 A).
// One CTA per home cell, launched interior cells first (the fullest cells start early and the
// light surface cells fill the tail), one warp per home octant. The 216 octants around the cell are
// staged in shared memory (in chunks if they exceed it); a warp's nb home atoms take nb i-slots
// and J = 32 / nb j-groups, each group walking a contiguous share of each of the 25 runs of
// neighbour octants (5 octants along x are adjacent in the staged order), so a warp reads at most
// J staged atoms per step. A pair is masked (r2 := inf) when r2 >= rcut^2 or when it is the atom
// itself (recognised by its place in the staged list), like the all-pairs cutoff variant, so every
// tested pair takes the same arithmetic as there.
#include "scmd_cells.cuh"

namespace scmd {

__global__ void k_cell_clear(const Dev d, int cond, int k_local) {
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    if (d.path == 2 && d.vslot && blockIdx.x == 0 && threadIdx.x == 0) *d.vslot = 0;  // FP64 lists
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.n_cells; c += gridDim.x * blockDim.x)
        d.cell_count[c] = 0;
}

// One thread per padded atom: its cell (from the FP64 state), an atomic slot in it, and at that
// slot its octant of the cell (the sign of its offset from the centre per axis) and the offset itself
// rounded once to the pass precision (in the cposg slots, free until the density pass).
template <int PREC> __global__ void k_cell_bin(const Dev d, int cond, int k_local) {
    using V4 = typename Tr<PREC>::V4;
    using R = typename Tr<PREC>::R;
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.npad) return;
    const int cl = d.cl_of_group[i >> 5];
    if (i - d.poff[cl] >= d.nreal[cl]) return;
    const CellGrid g = d.grid[cl];
    const double* o = d.origin + 3 * cl;
    const int np = d.npad;
    const double x = d.x[i], y = d.x[np + i], z = d.x[2 * np + i];
    const int cx = cell_axis(x - o[0], g), cy = cell_axis(y - o[1], g), cz = cell_axis(z - o[2], g);
    const int c = g.off + (cz * g.G + cy) * g.G + cx;
    const int slot = atomicAdd(d.cell_count + c, 1);
    if (slot >= kCellCap) {
        atomicOr(d.status, 2);
        return;
    }
    const double ox = o[0] + cell_centre(cx, g), oy = o[1] + cell_centre(cy, g), oz = o[2] + cell_centre(cz, g);
    const size_t k = (size_t)c * kCellCap + slot;
    d.cell_atoms[k] = i;
    d.cell_obyte[k] = (uint8_t)((x >= ox ? 1 : 0) | (y >= oy ? 2 : 0) | (z >= oz ? 4 : 0));
    V4 p;
    p.x = (R)(x - ox);
    p.y = (R)(y - oy);
    p.z = (R)(z - oz);
    p.w = R(0);
    reinterpret_cast<V4*>(d.cposg)[k] = p;
}

// One warp per cell: each atom's rank by (octant, atom index) is its place; its offset moves there
// (cposg -> cpos), and the first place of every octant (plus the count) goes to cell_oct.
template <int PREC> __global__ void k_cell_sort(const Dev d, int cond, int k_local) {
    using V4 = typename Tr<PREC>::V4;
    __shared__ int buf[kCellThreads / 32][kCellCap];
    __shared__ unsigned char boct[kCellThreads / 32][kCellCap];
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * (kCellThreads / 32) + w;
    if (c >= d.n_cells) return;
    const int n = min(d.cell_count[c], kCellCap);
    const size_t base = (size_t)c * kCellCap;
    int* a = d.cell_atoms + base;
    for (int k = lane; k < n; k += 32) {
        buf[w][k] = a[k];
        boct[w][k] = d.cell_obyte[base + k];
    }
    __syncwarp();
    if (lane < 9) {
        int cnt = 0;
        for (int q = 0; q < n; ++q) cnt += boct[w][q] < lane;
        d.cell_oct[c * 9 + lane] = cnt;
    }
    const V4* from = reinterpret_cast<const V4*>(d.cposg) + base;
    V4* cp = reinterpret_cast<V4*>(d.cpos) + base;
    for (int k = lane; k < n; k += 32) {
        const int e = buf[w][k], oc = boct[w][k];
        int r = 0;
        for (int q = 0; q < n; ++q) r += (boct[w][q] < oc) || (boct[w][q] == oc && buf[w][q] < e);
        a[r] = e;
        cp[r] = from[k];
    }
}

// ------------------------------------------------------------- density pass
template <int PREC, int SPECIAL, int SHIFT>
__global__ void __launch_bounds__(kCellThreads, PREC == 1 ? 5 : 2) k_cell_density(const Dev d, int obs) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    constexpr int TJ = CellChunk<PREC>::TJ;
    __shared__ V4 spos[TJ];
    __shared__ int s_src[kBoxN], s_cnt[kBoxN], s_pref[kBoxN + 1];
    __shared__ double part[8][32];
    __shared__ int2 s_runs[8][25];
    pdl_launch_dependents();
    pdl_wait();
    const int c = d.cell_order[blockIdx.x];
    if (d.cell_count[c] == 0) return;
    const int cl = d.cell_cl[c];
    const CellGrid g = d.grid[cl];
    const V4* cp = reinterpret_cast<const V4*>(d.cpos);
    const int M = octant_box(d, c, g, s_src, s_cnt, s_pref);
    const R rc2 = PREC == 1 ? (R)d.pot.rcut2f : (R)d.pot.rcut2, h = (R)g.h;
    const int mexp = d.pot.m;
    const int nblk = oct_blocks(d, c), lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int blk = 0; blk < nblk; ++blk) {
        const OctWarp q = oct_warp(d, c, blk * 32);
        const int slot = q.s0 + blk * 32 + q.is;
        const V4 pi = q.nb > 0 ? cp[(size_t)c * kCellCap + slot] : V4{};
        const int self = s_pref[q.home_t] + blk * 32 + q.is;
        f2sum facc = {0.f, 0.f};
        double racc = 0.0;
        int nin = 0;  // pairs inside rcut (the shifted form subtracts rcut^-m for each)
        for (int e0 = 0; e0 < M; e0 += TJ) {
            const int ne = min(TJ, M - e0);
            __syncthreads();
            gather_box(cp, s_src, s_pref, h, e0, ne, spos);
            __syncthreads();
            oct_runs(s_pref, q.o, e0, ne, s_runs[w]);
            if (!q.act) continue;
            const int selfl = self - e0;
#pragma unroll 1
            for (int run = 0; run < 25; ++run) {
                    const int2 ab = s_runs[w][run];
                    const int L = ab.y - ab.x, per = (L + q.J - 1) / q.J;
                    const int lo = ab.x + min(L, q.jg * per), hi = ab.x + min(L, q.jg * per + per);
                    R tacc = R(0);
#pragma unroll 4
                    for (int e = lo; e < hi; ++e) {
                        const V4 p = spos[e];
                        const R dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
                        R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                        const bool in = r2 < rc2 && e != selfl;
                        r2 = in ? r2 : big<R>();
                        if (SHIFT) nin += in;
                        if (SPECIAL) {
                            const R inv = inv_r2(r2);
                            tacc = fma(inv * inv, inv, tacc);
                        } else {
                            const R ir = inv_r(r2);
                            tacc += rpow(ir * ir, ir, mexp);
                        }
                    }
                    if (PREC == 1)
                        facc = f2_add(facc, (float)tacc);
                    else
                        racc += (double)tacc;
                }
        }
        if (PREC == 1) racc = (double)facc.hi + (double)facc.lo;
        if (SHIFT) racc -= (double)nin * d.pot.shm;
        part[w][lane] = racc;
        __syncwarp();
        if (q.nb > 0 && q.jg == 0) {
            double tot = part[w][q.is];
            for (int k = 1; k < q.J; ++k) tot += part[w][k * q.nb + q.is];
            const int i = d.cell_atoms[(size_t)c * kCellCap + slot];
            const double rho = tot * d.pot.am;
            d.rho[i] = rho;
            V4 p = pi;
            if (PREC == 1) {
                const float rf = (float)rho;
                float y = rsqrt_approx(rf);
                y = y * (1.5f - 0.5f * rf * y * y);  // one Newton step
                p.w = rho > 0.0 ? (float)d.pot.B6 * y : 0.0f;
            } else {
                p.w = rho > 0.0 ? d.pot.B6 / sqrt(rho) : 0.0;
            }
            reinterpret_cast<V4*>(d.cposg)[(size_t)c * kCellCap + slot] = p;
            if (obs) d.eatom[2 * i] = -d.pot.eps * d.pot.c * sqrt(rho);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------- force pass
// mode 0: forces; 1: forces and per-atom pair energies (observables of the current state);
// 2: MD step: second half kick, per-atom observables if due, then the first half of the next
// step unless this is the chunk's last step or the thermostat is Berendsen (whose kernel
// rescales and starts the next step).
template <int PREC, int SPECIAL, int ENERGY>
__global__ void __launch_bounds__(kCellThreads, PREC == 1 ? 5 : 2)
    k_cell_force(const Dev d, int mode, int k_local, int last) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    constexpr int TJ = CellChunk<PREC>::TJ;
    __shared__ V4 spos[TJ];
    __shared__ int s_src[kBoxN], s_cnt[kBoxN], s_pref[kBoxN + 1];
    __shared__ R partf[8][32][3];
    __shared__ double parte[ENERGY ? 8 : 1][32];
    __shared__ int2 s_runs[8][25];
    pdl_launch_dependents();
    pdl_wait();
    const int c = d.cell_order[blockIdx.x];
    if (d.cell_count[c] == 0) return;
    const int cl = d.cell_cl[c];
    const CellGrid g = d.grid[cl];
    const V4* pg = reinterpret_cast<const V4*>(d.cposg);
    const int M = octant_box(d, c, g, s_src, s_cnt, s_pref);
    const R A = PREC == 1 ? (R)d.pot.A9f : (R)d.pot.A9;
    const R rc2 = PREC == 1 ? (R)d.pot.rcut2f : (R)d.pot.rcut2, h = (R)g.h;
    const int nexp = d.pot.n, mexp = d.pot.m;
    const int nblk = oct_blocks(d, c), lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int blk = 0; blk < nblk; ++blk) {
        const OctWarp q = oct_warp(d, c, blk * 32);
        const int slot = q.s0 + blk * 32 + q.is;
        const V4 pi = q.nb > 0 ? pg[(size_t)c * kCellCap + slot] : V4{};
        const int self = s_pref[q.home_t] + blk * 32 + q.is;
        R fx = R(0), fy = R(0), fz = R(0);
        double ea = 0.0;
        int nin = 0;  // pairs inside rcut, counted with the energy (the shifted form)
        for (int e0 = 0; e0 < M; e0 += TJ) {
            const int ne = min(TJ, M - e0);
            __syncthreads();
            gather_box(pg, s_src, s_pref, h, e0, ne, spos);
            __syncthreads();
            oct_runs(s_pref, q.o, e0, ne, s_runs[w]);
            if (!q.act) continue;
            const int selfl = self - e0;
#pragma unroll 1
            for (int run = 0; run < 25; ++run) {
                    const int2 ab = s_runs[w][run];
                    const int L = ab.y - ab.x, per = (L + q.J - 1) / q.J;
                    const int lo = ab.x + min(L, q.jg * per), hi = ab.x + min(L, q.jg * per + per);
                    R sx = R(0), sy = R(0), sz = R(0), se = R(0);
#pragma unroll 4
                    for (int e = lo; e < hi; ++e) {
                        const V4 p = spos[e];
                        const R dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
                        R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                        const bool in = r2 < rc2 && e != selfl;
                        r2 = in ? r2 : big<R>();
                        if (ENERGY) nin += in;
                        const R ir = inv_r(r2);
                        const R inv = ir * ir;
                        R coef, rn;
                        if (SPECIAL) {
                            const R inv2 = inv * inv, inv4 = inv2 * inv2;
                            coef = inv4 * fma(A, inv * ir, -(pi.w + p.w));
                            rn = inv4 * ir;
                        } else {
                            rn = rpow(inv, ir, nexp);
                            const R rm = rpow(inv, ir, mexp);
                            coef = inv * (A * rn - (pi.w + p.w) * rm);
                        }
                        sx = fma(coef, dx, sx);
                        sy = fma(coef, dy, sy);
                        sz = fma(coef, dz, sz);
                        if (ENERGY) se += rn;
                    }
                    fx += sx;
                    fy += sy;
                    fz += sz;
                    if (ENERGY) ea += (double)se;
                }
        }
        partf[w][lane][0] = fx;
        partf[w][lane][1] = fy;
        partf[w][lane][2] = fz;
        if (ENERGY) parte[w][lane] = d.pot.shift ? ea - (double)nin * d.pot.shn : ea;
        __syncwarp();
        if (q.nb > 0 && q.jg == 0) {
            R Fx = partf[w][q.is][0], Fy = partf[w][q.is][1], Fz = partf[w][q.is][2];
            double Ep = ENERGY ? parte[w][q.is] : 0.0;
            for (int k = 1; k < q.J; ++k) {
                Fx += partf[w][k * q.nb + q.is][0];
                Fy += partf[w][k * q.nb + q.is][1];
                Fz += partf[w][k * q.nb + q.is][2];
                if (ENERGY) Ep += parte[w][k * q.nb + q.is];
            }
            const int i = d.cell_atoms[(size_t)c * kCellCap + slot];
            const int np = d.npad;
            R* fo = reinterpret_cast<R*>(d.f);
            fo[i] = Fx;
            fo[np + i] = Fy;
            fo[2 * np + i] = Fz;
            if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(d.status, 1);
            if (ENERGY) d.eatom[2 * i + 1] = Ep;
            if (mode == 2) {
                const Run& r = *d.run;
                const double hs = d.hs[i];
                const double vx = fma(hs, (double)Fx, d.v[i]);
                const double vy = fma(hs, (double)Fy, d.v[np + i]);
                const double vz = fma(hs, (double)Fz, d.v[2 * np + i]);
                d.v[i] = vx;
                d.v[np + i] = vy;
                d.v[2 * np + i] = vz;
                if (r.kind != 2) {  // Berendsen: the rescale kernel records and starts the step
                    if (ENERGY) {   // observables at the end of this step, before the next begins
                        for (int k = 0; k < 3; ++k) d.obs_x[3 * i + k] = d.x[k * np + i];
                        d.obs_v[3 * i] = vx;
                        d.obs_v[3 * i + 1] = vy;
                        d.obs_v[3 * i + 2] = vz;
                    }
                    if (!last)
                        begin_step<PREC>(d, r, i, cl, i - d.poff[cl], *d.step_base + k_local + 1, (double)Fx,
                                         (double)Fy, (double)Fz, k_local + 1);
                }
            }
        }
        __syncwarp();
    }
}

// Observable partials of one 32-atom group from the per-atom data of the cell path
// (the same per-group records and warp reductions as the all-pairs epilogues).
__global__ void k_cell_obs(const Dev d, int from_state, int with_velocity) {
    pdl_launch_dependents();
    pdl_wait();
    const int g = blockIdx.x, lane = threadIdx.x, i = g * 32 + lane;
    const int cl = d.cl_of_group[g];
    const bool real = i - d.poff[cl] < d.nreal[cl];
    const int np = d.npad;
    double m = 0.0, x = 0.0, y = 0.0, z = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    if (real) {
        m = d.mass[i];
        if (from_state) {
            x = d.x[i];
            y = d.x[np + i];
            z = d.x[2 * np + i];
            vx = d.v[i];
            vy = d.v[np + i];
            vz = d.v[2 * np + i];
        } else {
            x = d.obs_x[3 * i];
            y = d.obs_x[3 * i + 1];
            z = d.obs_x[3 * i + 2];
            vx = d.obs_v[3 * i];
            vy = d.obs_v[3 * i + 1];
            vz = d.obs_v[3 * i + 2];
        }
    }
    const double eemb = warp_sum(real ? d.eatom[2 * i] : 0.0);
    const double epair = warp_sum(real ? d.eatom[2 * i + 1] : 0.0);
    if (lane == 0) {
        d.part[(size_t)g * kObsFields + OF_EEMB] = eemb;
        d.part[(size_t)g * kObsFields + OF_EPAIR] = epair;
    }
    obs_position_partials(d, g, real, m, x, y, z, lane);
    if (with_velocity) obs_velocity_partials(d, g, real, m, x, y, z, vx, vy, vz, lane);
}

// Per-group sum m v^2 for the Berendsen rescale (the all-pairs force epilogue's reduction).
__global__ void k_cell_ke(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int g = blockIdx.x, lane = threadIdx.x, i = g * 32 + lane;
    const int cl = d.cl_of_group[g];
    const bool real = i - d.poff[cl] < d.nreal[cl];
    const int np = d.npad;
    const double m = real ? d.mass[i] : 0.0;
    const double vx = real ? d.v[i] : 0.0, vy = real ? d.v[np + i] : 0.0, vz = real ? d.v[2 * np + i] : 0.0;
    const double ke2 = warp_sum(real ? m * (vx * vx + vy * vy + vz * vz) : 0.0);
    if (lane == 0) d.ke_grp[g] = ke2;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_cell_build(const Dev& d, cudaStream_t s, int cond, int k_local, bool clear) {
    cudaError_t e = clear ? launch_ex(k_cell_clear, (d.n_cells + 255) / 256, 256, 0, 0, s, d, cond, k_local) : cudaSuccess;
    if (e != cudaSuccess) return e;
    e = d.prec == 1 ? launch_ex(k_cell_bin<1>, (d.npad + 255) / 256, 256, 0, 0, s, d, cond, k_local)
                    : launch_ex(k_cell_bin<0>, (d.npad + 255) / 256, 256, 0, 0, s, d, cond, k_local);
    if (e != cudaSuccess) return e;
    // MIXED neighbour lists: the quad build ranks each cell's atoms itself (by sub-cell, then index), from
    // the binned order, so the sort would not change any result
    if (d.path == 2 && d.prec == 1) return cudaSuccess;
    return d.prec == 1 ? launch_ex(k_cell_sort<1>, (d.n_cells + 7) / 8, kCellThreads, 0, 0, s, d, cond, k_local)
                       : launch_ex(k_cell_sort<0>, (d.n_cells + 7) / 8, kCellThreads, 0, 0, s, d, cond, k_local);
}

template <int PREC, int SHIFT>
static cudaError_t cell_density_s(const Dev& d, int obs, cudaStream_t s) {
    return d.pot.special ? launch_ex(k_cell_density<PREC, 1, SHIFT>, d.n_cells, kCellThreads, 0, 0, s, d, obs)
                         : launch_ex(k_cell_density<PREC, 0, SHIFT>, d.n_cells, kCellThreads, 0, 0, s, d, obs);
}

cudaError_t launch_cell_density(const Dev& d, int obs, cudaStream_t s) {
    const bool sh = d.pot.shift != 0;
    if (d.prec == 1) return sh ? cell_density_s<1, 1>(d, obs, s) : cell_density_s<1, 0>(d, obs, s);
    return sh ? cell_density_s<0, 1>(d, obs, s) : cell_density_s<0, 0>(d, obs, s);
}

template <int PREC, int ENERGY>
static cudaError_t cell_force_e(const Dev& d, int mode, int k, int last, cudaStream_t s) {
    return d.pot.special ? launch_ex(k_cell_force<PREC, 1, ENERGY>, d.n_cells, kCellThreads, 0, 0, s, d, mode, k, last)
                         : launch_ex(k_cell_force<PREC, 0, ENERGY>, d.n_cells, kCellThreads, 0, 0, s, d, mode, k, last);
}

cudaError_t launch_cell_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s) {
    const bool energy = (mode == 1) || (mode == 2 && (flags & 2));
    const int lst = flags & 1;
    if (d.prec == 1)
        return energy ? cell_force_e<1, 1>(d, mode, k_local, lst, s) : cell_force_e<1, 0>(d, mode, k_local, lst, s);
    return energy ? cell_force_e<0, 1>(d, mode, k_local, lst, s) : cell_force_e<0, 0>(d, mode, k_local, lst, s);
}

cudaError_t launch_cell_obs(const Dev& d, int from_state, int with_velocity, cudaStream_t s) {
    return launch_ex(k_cell_obs, d.ngroups, 32, 0, 0, s, d, from_state, with_velocity);
}

cudaError_t launch_cell_ke(const Dev& d, cudaStream_t s) { return launch_ex(k_cell_ke, d.ngroups, 32, 0, 0, s, d); }

}  // namespace scmd
