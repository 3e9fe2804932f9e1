// scmd_verlet.cu -- the neighbour-list path of the two pair passes (strict cutoff r < rcut).
//
// Each atom keeps the list of the atoms that were closer than rcut + skin when the lists were last
// built. As long as no atom has moved more than skin / 2 since, every pair closer than rcut is in
// the lists, so each pass tests only those entries (about (rcut + skin)^3 / rcut^3 of the pairs that
// count, against ~4x for the octants of the cell-list path). Per MD step:
//   k_v_anchor : every atom's offset from the centre of its cell at the last rebuild (its anchor),
//                in the pass precision, and the largest squared displacement since the rebuild;
//   rebuild, when that displacement exceeds (skin / 2)^2 (the kernels exit at once otherwise):
//     the cell build of the cell-list path (clear, bin, sort), then
//     k_v_build  : one CTA per home cell, the octant box staged in shared memory as in the
//                  cell-list passes; every atom closer than rcut + skin is appended to the home
//                  atom's list as (j << 6) | code, code = the cell offset a_i - a_j per axis + 1;
//     k_v_sort   : one warp per list, a bitonic sort by j;
//     k_v_commit : the new anchors, their offsets and the reference positions;
//   k_v_density, k_v_force : one thread per list (atoms in cell order, for cache locality).
// A pair's separation is (o_i - o_j) + (a_i - a_j) h, with o the anchor offsets and the shift taken
// from a per-cluster table of the 27 codes (exact in FP32: h is a binary32 value and |a_i - a_j| <= 1).
// Results do not depend on when the lists were built: a list holds every pair inside rcut in
// ascending j, a pair outside rcut is masked (r2 := inf) and adds an exact zero, and the pass-precision
// partial sums are folded every kSpanV pairs *inside rcut*. Resuming from a checkpoint (which rebuilds
// the lists) therefore reproduces an uninterrupted run bit for bit, as on the other paths.
#include "scmd_cells.cuh"

namespace scmd {

constexpr int kSpanV = 128;       // pairs inside rcut summed in the pass precision before a fold
constexpr int kVThreads = 256;
template <int PREC> struct BuildChunk;  // staged atoms per chunk of the list build (48 KB static limit)
template <> struct BuildChunk<1> { static constexpr int TJ = 1536; };
template <> struct BuildChunk<0> { static constexpr int TJ = 768; };

__device__ __forceinline__ int anchor_pack(int x, int y, int z) { return x | (y << 10) | (z << 20); }

// ---------------------------------------------------------------- every step
// Offsets from the anchor cells' centres, and the largest squared displacement since the rebuild
// under the step's parity (the other parity's slot is cleared for the next step).
template <int PREC> __global__ void k_v_anchor(const Dev d, int k_local) {
    using V4 = typename Tr<PREC>::V4;
    using R = typename Tr<PREC>::R;
    pdl_launch_dependents();
    pdl_wait();
    const int64_t step = *d.step_base + k_local;
    if (blockIdx.x == 0 && threadIdx.x == 0) d.vdmax[(step + 1) & 1] = 0u;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float dmax = 0.f;
    if (i < d.npad) {
        const int cl = d.cl_of_group[i >> 5];
        if (i - d.poff[cl] < d.nreal[cl]) {
            const CellGrid g = d.grid[cl];
            const double* o = d.origin + 3 * cl;
            const int np = d.npad, a = d.vanchor[i];
            const double x = d.x[i], y = d.x[np + i], z = d.x[2 * np + i];
            V4 p;
            p.x = (R)(x - (o[0] + cell_centre(a & 1023, g)));
            p.y = (R)(y - (o[1] + cell_centre((a >> 10) & 1023, g)));
            p.z = (R)(z - (o[2] + cell_centre(a >> 20, g)));
            p.w = R(0);
            reinterpret_cast<V4*>(d.vpos)[i] = p;
            const double ex = x - d.vxref[i], ey = y - d.vxref[np + i], ez = z - d.vxref[2 * np + i];
            dmax = (float)(ex * ex + ey * ey + ez * ez);
            if (!(dmax <= 3.0e38f)) dmax = 3.0e38f;  // non-finite positions force a rebuild
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, s));
    if ((threadIdx.x & 31) == 0 && dmax > 0.f) atomicMax(d.vdmax + (step & 1), __float_as_uint(dmax));
}

// ---------------------------------------------------------------- rebuild
// One CTA per home cell (interior first), one warp per home octant; every staged atom closer than
// rcut + skin goes into the home atom's list. The home cell's atoms take consecutive list slots.
template <int PREC>
__global__ void __launch_bounds__(kCellThreads, 2) k_v_build(const Dev d, int cond, int k_local) {
    using V4 = typename Tr<PREC>::V4;
    using R = typename Tr<PREC>::R;
    constexpr int TJ = BuildChunk<PREC>::TJ;
    __shared__ V4 spos[TJ];
    __shared__ int sidx[TJ];
    __shared__ unsigned char scode[TJ];
    __shared__ int s_src[kBoxN], s_cnt[kBoxN], s_pref[kBoxN + 1];
    __shared__ int2 s_runs[8][25];
    __shared__ int s_len[kCellCap];
    __shared__ int s_base;
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int c = d.cell_order[blockIdx.x];
    const int hc = min(d.cell_count[c], kCellCap);
    if (hc == 0) return;
    const int cl = d.cell_cl[c];
    const CellGrid g = d.grid[cl];
    const V4* cp = reinterpret_cast<const V4*>(d.cpos);
    const int M = octant_box(d, c, g, s_src, s_cnt, s_pref);
    for (int k = threadIdx.x; k < hc; k += blockDim.x) s_len[k] = 0;
    if (threadIdx.x == 0) s_base = atomicAdd(d.vslot, hc);
    __syncthreads();
    const int base = s_base, ns = d.nslot;
    for (int k = threadIdx.x; k < hc; k += blockDim.x) d.vorder[base + k] = d.cell_atoms[(size_t)c * kCellCap + k];
    const R rl2 = (R)d.vrl2, h = (R)g.h;
    const int nblk = oct_blocks(d, c), w = threadIdx.x >> 5;
    bool overflow = false;
    for (int blk = 0; blk < nblk; ++blk) {
        const OctWarp q = oct_warp(d, c, blk * 32);
        const int k_home = q.s0 + blk * 32 + q.is;  // the home atom's place in its cell
        const V4 pi = q.nb > 0 ? cp[(size_t)c * kCellCap + k_home] : V4{};
        const int self = s_pref[q.home_t] + blk * 32 + q.is;
        int* list = d.vlist + base + k_home;
        for (int e0 = 0; e0 < M; e0 += TJ) {
            const int ne = min(TJ, M - e0);
            __syncthreads();
            for (int t = threadIdx.x; t < kBoxN; t += blockDim.x) {  // stage positions, atoms and codes
                const int a = max(s_pref[t], e0), b = min(s_pref[t + 1], e0 + ne);
                const int dx = (t % kBox) / 2 - 1, dy = ((t / kBox) % kBox) / 2 - 1, dz = (t / (kBox * kBox)) / 2 - 1;
                const R sx = (R)dx * h, sy = (R)dy * h, sz = (R)dz * h;
                const unsigned char code = (unsigned char)((1 - dx) | ((1 - dy) << 2) | ((1 - dz) << 4));
                for (int e = a; e < b; ++e) {
                    const int src = s_src[t] + (e - s_pref[t]);
                    V4 p = cp[src];
                    p.x += sx;
                    p.y += sy;
                    p.z += sz;
                    spos[e - e0] = p;
                    sidx[e - e0] = d.cell_atoms[src];
                    scode[e - e0] = code;
                }
            }
            __syncthreads();
            oct_runs(s_pref, q.o, e0, ne, s_runs[w]);
            if (!q.act) continue;
            const int selfl = self - e0;
            for (int run = 0; run < 25; ++run) {
                const int2 ab = s_runs[w][run];
                const int L = ab.y - ab.x, per = (L + q.J - 1) / q.J;
                const int lo = ab.x + min(L, q.jg * per), hi = ab.x + min(L, q.jg * per + per);
                for (int e = lo; e < hi; ++e) {
                    const V4 p = spos[e];
                    const R dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
                    const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    if (r2 < rl2 && e != selfl) {
                        const int slot = atomicAdd(&s_len[k_home], 1);
                        if (slot < kVMax)
                            list[(size_t)slot * ns] = (sidx[e] << 6) | scode[e];
                        else
                            overflow = true;
                    }
                }
            }
        }
    }
    if (overflow) atomicOr(d.status, 4);
    __syncthreads();
    for (int k = threadIdx.x; k < hc; k += blockDim.x) d.vcount[base + k] = min(s_len[k], kVMax);
}

// One warp per list: a bitonic sort of its entries (by j, which sits in the high bits).
__global__ void __launch_bounds__(kVThreads) k_v_sort(const Dev d, int cond, int k_local) {
    __shared__ uint32_t buf[kVThreads / 32][kVMax];
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * (kVThreads / 32) + w;
    if (s >= d.nslot) return;
    const int n = d.vcount[s], ns = d.nslot;
    int P = 32;
    while (P < n) P <<= 1;
    uint32_t* b = buf[w];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(d.vlist) + s;
    for (int e = lane; e < P; e += 32) b[e] = e < n ? src[(size_t)e * ns] : 0xffffffffu;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = lane; e < P; e += 32) {
                const int f = e ^ j;
                if (f > e) {
                    const uint32_t x = b[e], y = b[f];
                    if ((x > y) == ((e & k) == 0)) {
                        b[e] = y;
                        b[f] = x;
                    }
                }
            }
            __syncwarp();
        }
    uint32_t* dst = reinterpret_cast<uint32_t*>(d.vlist) + s;
    for (int e = lane; e < n; e += 32) dst[(size_t)e * ns] = b[e];
}

// New anchors (the cell each atom was binned into by this rebuild), their offsets and the positions
// the next displacements are measured from.
template <int PREC> __global__ void k_v_commit(const Dev d, int cond, int k_local) {
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
    d.vanchor[i] = anchor_pack(cx, cy, cz);
    d.vxref[i] = x;
    d.vxref[np + i] = y;
    d.vxref[2 * np + i] = z;
    V4 p;
    p.x = (R)(x - (o[0] + cell_centre(cx, g)));
    p.y = (R)(y - (o[1] + cell_centre(cy, g)));
    p.z = (R)(z - (o[2] + cell_centre(cz, g)));
    p.w = R(0);
    reinterpret_cast<V4*>(d.vpos)[i] = p;
}

// ---------------------------------------------------------------- passes
template <int PREC, int SPECIAL>
__global__ void __launch_bounds__(kVThreads) k_v_density(const Dev d, int obs) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    pdl_launch_dependents();
    pdl_wait();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.nslot) return;
    const int i = d.vorder[s], n = d.vcount[s], ns = d.nslot;
    const int cl = d.cl_of_group[i >> 5];
    const V4* vp = reinterpret_cast<const V4*>(d.vpos);
    const V4* sh = reinterpret_cast<const V4*>(d.vshift) + 64 * cl;
    const V4 pi = vp[i];
    const R rc2 = (R)d.pot.rcut2;
    const int mexp = d.pot.m;
    const int* lst = d.vlist + s;
    f2sum facc = {0.f, 0.f};
    double racc = 0.0;
    R tacc = R(0);
    int cnt = 0;
#pragma unroll 4
    for (int e = 0; e < n; ++e) {
        const uint32_t q = (uint32_t)lst[(size_t)e * ns];
        const V4 pj = vp[q >> 6], t = sh[q & 63];
        const R dx = (pi.x - pj.x) + t.x, dy = (pi.y - pj.y) + t.y, dz = (pi.z - pj.z) + t.z;
        R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const bool in = r2 < rc2;
        r2 = in ? r2 : big<R>();
        if (SPECIAL) {
            const R inv = inv_r2(r2);
            tacc = fma(inv * inv, inv, tacc);
        } else {
            const R ir = inv_r(r2);
            tacc += rpow(ir * ir, ir, mexp);
        }
        cnt += in;
        if (cnt == kSpanV) {
            if (PREC == 1)
                facc = f2_add(facc, (float)tacc);
            else
                racc += (double)tacc;
            tacc = R(0);
            cnt = 0;
        }
    }
    if (PREC == 1) {
        facc = f2_add(facc, (float)tacc);
        racc = (double)facc.hi + (double)facc.lo;
    } else {
        racc += (double)tacc;
    }
    const double rho = racc * d.pot.am;
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
    reinterpret_cast<V4*>(d.vposg)[i] = p;
    if (obs) d.eatom[2 * i] = -d.pot.eps * d.pot.c * sqrt(rho);
}

// mode 0: forces; 1: forces and per-atom pair energies; 2: MD step (second half kick, per-atom
// observables if due, then the first half of the next step unless last or Berendsen).
template <int PREC, int SPECIAL, int ENERGY>
__global__ void __launch_bounds__(kVThreads) k_v_force(const Dev d, int mode, int k_local, int last) {
    using R = typename Tr<PREC>::R;
    using V4 = typename Tr<PREC>::V4;
    pdl_launch_dependents();
    pdl_wait();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.nslot) return;
    const int i = d.vorder[s], n = d.vcount[s], ns = d.nslot;
    const int cl = d.cl_of_group[i >> 5];
    const V4* vp = reinterpret_cast<const V4*>(d.vposg);
    const V4* sh = reinterpret_cast<const V4*>(d.vshift) + 64 * cl;
    const V4 pi = vp[i];
    const R A = (R)d.pot.A9;
    const R rc2 = (R)d.pot.rcut2;
    const int nexp = d.pot.n, mexp = d.pot.m;
    const int* lst = d.vlist + s;
    R fx = R(0), fy = R(0), fz = R(0), sx = R(0), sy = R(0), sz = R(0), se = R(0);
    double ea = 0.0;
    int cnt = 0;
#pragma unroll 4
    for (int e = 0; e < n; ++e) {
        const uint32_t q = (uint32_t)lst[(size_t)e * ns];
        const V4 pj = vp[q >> 6], t = sh[q & 63];
        const R dx = (pi.x - pj.x) + t.x, dy = (pi.y - pj.y) + t.y, dz = (pi.z - pj.z) + t.z;
        R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const bool in = r2 < rc2;
        r2 = in ? r2 : big<R>();
        const R ir = inv_r(r2);
        const R inv = ir * ir;
        R coef, rn;
        if (SPECIAL) {
            const R inv2 = inv * inv, inv4 = inv2 * inv2;
            coef = inv4 * fma(A, inv * ir, -(pi.w + pj.w));
            rn = inv4 * ir;
        } else {
            rn = rpow(inv, ir, nexp);
            const R rm = rpow(inv, ir, mexp);
            coef = inv * (A * rn - (pi.w + pj.w) * rm);
        }
        sx = fma(coef, dx, sx);
        sy = fma(coef, dy, sy);
        sz = fma(coef, dz, sz);
        if (ENERGY) se += rn;
        cnt += in;
        if (cnt == kSpanV) {
            fx += sx;
            fy += sy;
            fz += sz;
            sx = sy = sz = R(0);
            if (ENERGY) {
                ea += (double)se;
                se = R(0);
            }
            cnt = 0;
        }
    }
    const R Fx = fx + sx, Fy = fy + sy, Fz = fz + sz;
    const double Ep = ea + (double)se;
    const int np = d.npad;
    R* fo = reinterpret_cast<R*>(d.f);
    fo[i] = Fx;
    fo[np + i] = Fy;
    fo[2 * np + i] = Fz;
    if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(d.status, 1);
    if (ENERGY) d.eatom[2 * i + 1] = Ep;
    if (mode != 2) return;
    const Run& r = *d.run;
    const double hs = d.hs[i];
    const double vx = fma(hs, (double)Fx, d.v[i]);
    const double vy = fma(hs, (double)Fy, d.v[np + i]);
    const double vz = fma(hs, (double)Fz, d.v[2 * np + i]);
    d.v[i] = vx;
    d.v[np + i] = vy;
    d.v[2 * np + i] = vz;
    if (r.kind == 2) return;  // Berendsen: the rescale kernel records and starts the step
    if (ENERGY) {             // observables at the end of this step, before the next begins
        for (int k = 0; k < 3; ++k) d.obs_x[3 * i + k] = d.x[k * np + i];
        d.obs_v[3 * i] = vx;
        d.obs_v[3 * i + 1] = vy;
        d.obs_v[3 * i + 2] = vz;
    }
    if (!last)
        begin_step<PREC>(d, r, i, cl, i - d.poff[cl], *d.step_base + k_local + 1, (double)Fx, (double)Fy,
                         (double)Fz, k_local + 1);
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_v_anchor(const Dev& d, int k_local, cudaStream_t s) {
    const int grid = (d.npad + kVThreads - 1) / kVThreads;
    return d.prec == 1 ? launch_ex(k_v_anchor<1>, grid, kVThreads, 0, 0, s, d, k_local)
                       : launch_ex(k_v_anchor<0>, grid, kVThreads, 0, 0, s, d, k_local);
}

cudaError_t launch_v_rebuild(const Dev& d, int cond, int k_local, cudaStream_t s) {
    cudaError_t e = d.prec == 1 ? launch_ex(k_v_build<1>, d.n_cells, kCellThreads, 0, 0, s, d, cond, k_local)
                                : launch_ex(k_v_build<0>, d.n_cells, kCellThreads, 0, 0, s, d, cond, k_local);
    if (e != cudaSuccess) return e;
    e = launch_ex(k_v_sort, (d.nslot + 7) / 8, kVThreads, 0, 0, s, d, cond, k_local);
    if (e != cudaSuccess) return e;
    const int grid = (d.npad + kVThreads - 1) / kVThreads;
    return d.prec == 1 ? launch_ex(k_v_commit<1>, grid, kVThreads, 0, 0, s, d, cond, k_local)
                       : launch_ex(k_v_commit<0>, grid, kVThreads, 0, 0, s, d, cond, k_local);
}

cudaError_t launch_v_density(const Dev& d, int obs, cudaStream_t s) {
    const int grid = (d.nslot + kVThreads - 1) / kVThreads;
    const bool sp = d.pot.special != 0;
    if (d.prec == 1)
        return sp ? launch_ex(k_v_density<1, 1>, grid, kVThreads, 0, 0, s, d, obs)
                  : launch_ex(k_v_density<1, 0>, grid, kVThreads, 0, 0, s, d, obs);
    return sp ? launch_ex(k_v_density<0, 1>, grid, kVThreads, 0, 0, s, d, obs)
              : launch_ex(k_v_density<0, 0>, grid, kVThreads, 0, 0, s, d, obs);
}

template <int PREC, int ENERGY>
static cudaError_t v_force_e(const Dev& d, int mode, int k, int last, cudaStream_t s) {
    const int grid = (d.nslot + kVThreads - 1) / kVThreads;
    return d.pot.special ? launch_ex(k_v_force<PREC, 1, ENERGY>, grid, kVThreads, 0, 0, s, d, mode, k, last)
                         : launch_ex(k_v_force<PREC, 0, ENERGY>, grid, kVThreads, 0, 0, s, d, mode, k, last);
}

cudaError_t launch_v_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s) {
    const bool energy = (mode == 1) || (mode == 2 && (flags & 2));
    const int lst = flags & 1;
    if (d.prec == 1)
        return energy ? v_force_e<1, 1>(d, mode, k_local, lst, s) : v_force_e<1, 0>(d, mode, k_local, lst, s);
    return energy ? v_force_e<0, 1>(d, mode, k_local, lst, s) : v_force_e<0, 0>(d, mode, k_local, lst, s);
}

}  // namespace scmd
