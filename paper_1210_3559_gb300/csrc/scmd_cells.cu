// scmd_cells.cu -- the cell-list path of the two pair passes (strict cutoff r < rcut).
//
// The paper evaluates every pair and names efficient cutoff schemes as work in progress
// (Sec. II). With rcut > 0 a context may instead give each cluster a cubic grid of G^3 cells of
// side h >= rcut, fixed when the context is created: the cube [-E, E)^3 around the cluster's
// origin (the centre of mass that the MIXED pair coordinates are measured from), with E a
// margin beyond the cluster's radius. Atoms outside the cube are clamped into its border
// cells; clamping is monotone per axis, so two atoms closer than rcut still sit in the same or
// in adjacent cells. Per MD step:
//   k_cell_clear, k_cell_bin : atoms binned into cells of fixed capacity (atomic slots;
//                              an overflow sets status bit 1, reported by the host);
//   k_cell_sort              : each cell's list sorted by atom index, so the order of every
//                              sum below and hence the results are independent of the order in
//                              which the atomic slots were taken;
//   k_cell_density           : rho_i over the 27 neighbour cells (Eq. 2 with the cutoff);
//   k_cell_force             : F_i over the 27 neighbour cells (-grad of Eq. 1 with the
//                              cutoff), then the integrator step of the all-pairs path.
// Pair coordinates are relative to cell centres: when the atoms are binned, each cell stores its
// atoms' offsets x - centre (rounded once from the FP64 state to the pass precision), and a CTA
// moves a neighbour cell's offsets to its own centre by adding (k - l) h, which is exact in FP32
// (h is a binary32 value). In MIXED mode a coordinate is then off by at most about
// ulp(1.5 h) ~ 5e-7 A whatever the cluster's size, where offsets from one origin per cluster
// would carry ulp(R) (about 2e-6 A at R = 50 A).
// One CTA per home cell, launched interior cells first (the fullest cells start early and the
// light surface cells fill the tail). The atoms of the 27 neighbour cells are gathered into shared
// memory in chunks; the home cell's nb atoms (nb <= 256) take nb i-slots and J = 256 / nb j-groups,
// each walking a contiguous share of every chunk, so a warp reads one or two staged atoms per step
// for up to 32 i-atoms. A pair is masked (r2 := inf) when r2 >= rcut^2 or when it is the atom itself
// (recognised by its place in the staged list), like the all-pairs cutoff variant, so every tested
// pair takes the same arithmetic as there.
#include "scmd_device.cuh"

namespace scmd {

constexpr int kCellThreads = 256;
constexpr int kSpan = 128;  // pair terms summed in the pass precision before folding into the wider sums
template <int PREC> struct CellChunk;
template <> struct CellChunk<1> { static constexpr int TJ = 2048; };  // 32 KB of float4
template <> struct CellChunk<0> { static constexpr int TJ = 1024; };  // 32 KB of double4

// Cell index along one axis of a coordinate relative to the origin. fmin/fmax come before the
// conversion: far or non-finite coordinates land in a border cell.
__device__ __forceinline__ int cell_axis(double rel, const CellGrid& g) {
    return (int)fmin(fmax(floor((rel + g.E) / g.h), 0.0), (double)(g.G - 1));
}
// Centre of cell k along one axis, relative to the origin (exact: h is a binary32 value).
__device__ __forceinline__ double cell_centre(int k, const CellGrid& g) { return -g.E + (k + 0.5) * g.h; }

__global__ void k_cell_clear(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.n_cells; c += gridDim.x * blockDim.x)
        d.cell_count[c] = 0;
}

// One thread per padded atom: its cell (from the FP64 state), and an atomic slot in it.
__global__ void k_cell_bin(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.npad) return;
    const int cl = d.cl_of_group[i >> 5];
    if (i - d.poff[cl] >= d.nreal[cl]) return;
    const CellGrid g = d.grid[cl];
    const double* o = d.origin + 3 * cl;
    const int np = d.npad;
    const int cx = cell_axis(d.x[i] - o[0], g), cy = cell_axis(d.x[np + i] - o[1], g);
    const int cz = cell_axis(d.x[2 * np + i] - o[2], g);
    const int c = g.off + (cz * g.G + cy) * g.G + cx;
    const int slot = atomicAdd(d.cell_count + c, 1);
    if (slot < kCellCap)
        d.cell_atoms[(size_t)c * kCellCap + slot] = i;
    else
        atomicOr(d.status, 2);
}

// One warp per cell: each entry's rank among the cell's (distinct) atom indices is its place;
// the atom's offset from the cell centre is stored at the same place.
template <int PREC> __global__ void k_cell_sort(const Dev d) {
    using V4 = typename Tr<PREC>::V4;
    __shared__ int buf[kCellThreads / 32][kCellCap];
    pdl_launch_dependents();
    pdl_wait();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * (kCellThreads / 32) + w;
    if (c >= d.n_cells) return;
    const int n = min(d.cell_count[c], kCellCap);
    int* a = d.cell_atoms + (size_t)c * kCellCap;
    for (int k = lane; k < n; k += 32) buf[w][k] = a[k];
    __syncwarp();
    if (n == 0) return;
    const int cl = d.cell_cl[c];
    const CellGrid g = d.grid[cl];
    const int loc = c - g.off, np = d.npad;
    const double* o = d.origin + 3 * cl;
    const double ox = o[0] + cell_centre(loc % g.G, g), oy = o[1] + cell_centre((loc / g.G) % g.G, g);
    const double oz = o[2] + cell_centre(loc / (g.G * g.G), g);
    V4* cp = reinterpret_cast<V4*>(d.cpos) + (size_t)c * kCellCap;
    for (int k = lane; k < n; k += 32) {
        const int e = buf[w][k];
        int r = 0;
        for (int q = 0; q < n; ++q) r += buf[w][q] < e;
        a[r] = e;
        using R = typename Tr<PREC>::R;
        V4 p;
        p.x = (R)(d.x[e] - ox);
        p.y = (R)(d.x[np + e] - oy);
        p.z = (R)(d.x[2 * np + e] - oz);
        p.w = R(0);
        cp[r] = p;
    }
}

// The 27 neighbour cells of home cell c (those off the grid count as empty): their ids and
// the prefix sums of their counts. Every thread of the CTA calls this.
__device__ __forceinline__ int stencil(const Dev& d, int c, int cl, int* scell, int* pref) {
    const CellGrid g = d.grid[cl];
    const int loc = c - g.off, cx = loc % g.G, cy = (loc / g.G) % g.G, cz = loc / (g.G * g.G);
    if (threadIdx.x < 27) {
        const int k = threadIdx.x;
        const int x = cx + k % 3 - 1, y = cy + (k / 3) % 3 - 1, z = cz + k / 9 - 1;
        int id = -1, n = 0;
        if (x >= 0 && x < g.G && y >= 0 && y < g.G && z >= 0 && z < g.G) {
            id = g.off + (z * g.G + y) * g.G + x;
            n = min(d.cell_count[id], kCellCap);
        }
        scell[k] = id;
        pref[k + 1] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        pref[0] = 0;
        for (int k = 0; k < 27; ++k) pref[k + 1] += pref[k];
    }
    __syncthreads();
    return pref[27];
}

// Stage entries e0 .. e0 + ne - 1 of the neighbour list: cell-slot data from src (offsets from
// the neighbour cell's centre), moved to the home cell's centre by the exact (k - l) h.
template <class V4, class R>
__device__ __forceinline__ void gather(const V4* __restrict__ src, const int* scell, const int* pref, R h, int e0,
                                       int ne, V4* spos) {
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const int q = e0 + e;
        int k = 0;
        while (pref[k + 1] <= q) ++k;
        V4 p = src[(size_t)scell[k] * kCellCap + (q - pref[k])];
        p.x += (R)(k % 3 - 1) * h;
        p.y += (R)((k / 3) % 3 - 1) * h;
        p.z += (R)(k / 9 - 1) * h;
        spos[e] = p;
    }
}

// ------------------------------------------------------------- density pass
template <int PREC, int SPECIAL>
__global__ void __launch_bounds__(kCellThreads, PREC == 1 ? 5 : 2) k_cell_density(const Dev d, int obs) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    constexpr int TJ = CellChunk<PREC>::TJ;
    __shared__ V4 spos[TJ];
    __shared__ int scell[27], pref[28];
    __shared__ double part[kCellThreads];
    pdl_launch_dependents();
    pdl_wait();
    const int c = d.cell_order[blockIdx.x];
    const int hc = min(d.cell_count[c], kCellCap);
    if (hc == 0) return;
    const int cl = d.cell_cl[c];
    const V4* cp = reinterpret_cast<const V4*>(d.cpos);
    const int M = stencil(d, c, cl, scell, pref);
    const R rc2 = (R)d.pot.rcut2, h = (R)d.grid[cl].h;
    const int mexp = d.pot.m;
    const int* home = d.cell_atoms + (size_t)c * kCellCap;
    for (int r0 = 0; r0 < hc; r0 += kCellThreads) {
        const int nb = min(kCellThreads, hc - r0), J = kCellThreads / nb;
        const int t = threadIdx.x, is = t % nb, jg = t / nb;
        const bool act = jg < J;
        const int i = home[r0 + is];
        const int self = pref[13] + r0 + is;  // the home cell is stencil entry 13
        const V4 pi = cp[(size_t)c * kCellCap + r0 + is];
        f2sum facc = {0.f, 0.f};
        double racc = 0.0;
        for (int e0 = 0; e0 < M; e0 += TJ) {
            const int ne = min(TJ, M - e0);
            __syncthreads();
            gather(cp, scell, pref, h, e0, ne, spos);
            __syncthreads();
            if (!act) continue;
            // this j-group's contiguous share of the chunk, summed in spans of kSpan terms
            const int per = (ne + J - 1) / J, lo = min(ne, jg * per), hi = min(ne, lo + per);
            const int selfl = self - e0;
            for (int b = lo; b < hi; b += kSpan) {
                const int stop = min(hi, b + kSpan);
                R tacc = R(0);
#pragma unroll 4
                for (int e = b; e < stop; ++e) {
                    const V4 p = spos[e];
                    const R dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
                    R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    r2 = (r2 < rc2 && e != selfl) ? r2 : big<R>();
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
        part[t] = racc;
        __syncthreads();
        if (jg == 0) {
            double tot = part[is];
            for (int g = 1; g < J; ++g) tot += part[g * nb + is];
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
            reinterpret_cast<V4*>(d.cposg)[(size_t)c * kCellCap + r0 + is] = p;
            if (obs) d.eatom[2 * i] = -d.pot.eps * d.pot.c * sqrt(rho);
        }
    }
}

// ------------------------------------------------------------- force pass
// mode 0: forces; 1: forces and per-atom pair energies (observables of the current state);
// 2: MD step: second half kick, per-atom observables if due, then the first half of the next
// step unless this is the chunk's last step or the thermostat is Berendsen (whose kernel
// rescales and starts the next step).
template <int PREC, int SPECIAL, int ENERGY>
__global__ void __launch_bounds__(kCellThreads, PREC == 1 ? 5 : 2) k_cell_force(const Dev d, int mode, int k_local, int last) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    constexpr int TJ = CellChunk<PREC>::TJ;
    __shared__ V4 spos[TJ];
    __shared__ int scell[27], pref[28];
    __shared__ R partf[kCellThreads][3];
    __shared__ double parte[ENERGY ? kCellThreads : 1];
    pdl_launch_dependents();
    pdl_wait();
    const int c = d.cell_order[blockIdx.x];
    const int hc = min(d.cell_count[c], kCellCap);
    if (hc == 0) return;
    const int cl = d.cell_cl[c];
    const V4* pg = reinterpret_cast<const V4*>(d.cposg);
    const int M = stencil(d, c, cl, scell, pref);
    const R A = (R)d.pot.A9;
    const R rc2 = (R)d.pot.rcut2, h = (R)d.grid[cl].h;
    const int nexp = d.pot.n, mexp = d.pot.m;
    const int* home = d.cell_atoms + (size_t)c * kCellCap;
    for (int r0 = 0; r0 < hc; r0 += kCellThreads) {
        const int nb = min(kCellThreads, hc - r0), J = kCellThreads / nb;
        const int t = threadIdx.x, is = t % nb, jg = t / nb;
        const bool act = jg < J;
        const int i = home[r0 + is];
        const int self = pref[13] + r0 + is;
        const V4 pi = pg[(size_t)c * kCellCap + r0 + is];
        R fx = R(0), fy = R(0), fz = R(0);
        double ea = 0.0;
        for (int e0 = 0; e0 < M; e0 += TJ) {
            const int ne = min(TJ, M - e0);
            __syncthreads();
            gather(pg, scell, pref, h, e0, ne, spos);
            __syncthreads();
            if (!act) continue;
            const int per = (ne + J - 1) / J, lo = min(ne, jg * per), hi = min(ne, lo + per);
            const int selfl = self - e0;
            for (int b = lo; b < hi; b += kSpan) {
                const int stop = min(hi, b + kSpan);
                R sx = R(0), sy = R(0), sz = R(0), se = R(0);
#pragma unroll 4
                for (int e = b; e < stop; ++e) {
                    const V4 p = spos[e];
                    const R dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
                    R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    r2 = (r2 < rc2 && e != selfl) ? r2 : big<R>();
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
        partf[t][0] = fx;
        partf[t][1] = fy;
        partf[t][2] = fz;
        if (ENERGY) parte[t] = ea;
        __syncthreads();
        if (jg != 0) continue;
        R Fx = partf[is][0], Fy = partf[is][1], Fz = partf[is][2];
        double Ep = ENERGY ? parte[is] : 0.0;
        for (int g = 1; g < J; ++g) {
            Fx += partf[g * nb + is][0];
            Fy += partf[g * nb + is][1];
            Fz += partf[g * nb + is][2];
            if (ENERGY) Ep += parte[g * nb + is];
        }
        const int np = d.npad;
        R* fo = reinterpret_cast<R*>(d.f);
        fo[i] = Fx;
        fo[np + i] = Fy;
        fo[2 * np + i] = Fz;
        if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(d.status, 1);
        if (ENERGY) d.eatom[2 * i + 1] = Ep;
        if (mode != 2) continue;
        const Run& r = *d.run;
        const double hs = d.hs[i];
        const double vx = fma(hs, (double)Fx, d.v[i]);
        const double vy = fma(hs, (double)Fy, d.v[np + i]);
        const double vz = fma(hs, (double)Fz, d.v[2 * np + i]);
        d.v[i] = vx;
        d.v[np + i] = vy;
        d.v[2 * np + i] = vz;
        if (r.kind == 2) continue;  // Berendsen: the rescale kernel records and starts the step
        if (ENERGY) {               // observables at the end of this step, before the next begins
            for (int k = 0; k < 3; ++k) d.obs_x[3 * i + k] = d.x[k * np + i];
            d.obs_v[3 * i] = vx;
            d.obs_v[3 * i + 1] = vy;
            d.obs_v[3 * i + 2] = vz;
        }
        if (!last)
            begin_step<PREC>(d, r, i, cl, i - d.poff[cl], *d.step_base + k_local + 1, (double)Fx, (double)Fy,
                             (double)Fz, k_local + 1);
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
cudaError_t launch_cell_build(const Dev& d, cudaStream_t s) {
    cudaError_t e = launch_ex(k_cell_clear, (d.n_cells + 255) / 256, 256, 0, 0, s, d);
    if (e != cudaSuccess) return e;
    e = launch_ex(k_cell_bin, (d.npad + 255) / 256, 256, 0, 0, s, d);
    if (e != cudaSuccess) return e;
    return d.prec == 1 ? launch_ex(k_cell_sort<1>, (d.n_cells + 7) / 8, kCellThreads, 0, 0, s, d)
                       : launch_ex(k_cell_sort<0>, (d.n_cells + 7) / 8, kCellThreads, 0, 0, s, d);
}

cudaError_t launch_cell_density(const Dev& d, int obs, cudaStream_t s) {
    const bool sp = d.pot.special != 0;
    if (d.prec == 1)
        return sp ? launch_ex(k_cell_density<1, 1>, d.n_cells, kCellThreads, 0, 0, s, d, obs)
                  : launch_ex(k_cell_density<1, 0>, d.n_cells, kCellThreads, 0, 0, s, d, obs);
    return sp ? launch_ex(k_cell_density<0, 1>, d.n_cells, kCellThreads, 0, 0, s, d, obs)
              : launch_ex(k_cell_density<0, 0>, d.n_cells, kCellThreads, 0, 0, s, d, obs);
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
