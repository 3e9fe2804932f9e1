// scmd_verlet.cu -- the neighbour-list path of the two pair passes (strict cutoff r < rcut), FP64.
// (MIXED lists are lists of atom quads: scmd_quads.cu.)
//
// Each atom keeps the list of the atoms with a higher index that were closer than rcut + skin when
// the lists were last built (a half list: every pair once, Newton's third law gives the partner's
// share). As long as no atom has moved more than skin / 2 since, every pair closer than rcut is in
// the lists, so each pass computes only those entries (about (rcut + skin)^3 / rcut^3 of the pairs
// that count, halved, against ~4x for the octants of the cell-list path). Per MD step:
//   k_v_pos    : every atom's pass coordinates, by list slot, and the largest squared displacement
//                since the last rebuild;
//   rebuild, when that displacement exceeds the trigger (the kernels exit at once otherwise):
//     the cell build of the cell-list path (clear, bin, sort), then
//     k_v_build  : one CTA per home cell, the octant box staged in shared memory as in the
//                  cell-list passes; every atom closer than rcut + skin is appended to the home
//                  atom's list. The home cell's atoms take consecutive slots (cell order);
//     k_v_sort   : one warp per list, a bitonic sort by (j mod kVLanes, j), the atoms turned into
//                  their slots, the ends of the kVLanes sub-lists, and each entry appended to the
//                  partner's reverse list;
//     k_v_rsort  : one warp per slot, its reverse list sorted by (lower atom mod kVLanes, lower atom);
//     k_v_commit : the pass coordinates in the new slot order and the reference positions;
//   k_v_compact : one warp per atom, every step: the list entries inside rcut now, in list order;
//   k_v_density, k_v_force : kVLanes threads per atom, thread t over compacted entries t, t + kVLanes,
//                  ...; each pair term goes into the atom's own sum and into a buffer at the entry's
//                  place;
//   k_v_dgather, k_v_fgather : kVLanes threads per atom, its own sum plus (or, for forces, minus)
//                  the buffered terms of its reverse list; then, one warp per 32 atoms, rho and g, or
//                  the integrator step.
// The passes read the positions themselves (by slot).
// Results do not depend on when the lists were built: the compacted entries are the pairs inside
// rcut in the order of the keys (j mod kVLanes, j), a function of the positions alone, so which
// thread takes an entry and in which order is fixed too; partial sums are folded every kSpanV
// entries; the kVLanes partials are added in a fixed tree; and the reverse list is summed in
// ascending order of the lower atom, split by its residue class in the same way (entries outside
// rcut this step are skipped by their flag). Resuming from a checkpoint (which rebuilds
// the lists) therefore reproduces an uninterrupted run bit for bit, as on the other paths.
#include "scmd_cells.cuh"

namespace scmd {

constexpr int kSpanV = 64;  // pairs inside rcut a thread sums in the pass precision before a fold
constexpr int kVThreads = 256;
constexpr int kBuildTJ = 1536;  // staged atoms per chunk of the list build (float4 + index: 30 KB)
static_assert(kVLog >= 1 && kVLog <= 4, "an atom's threads must sit in one warp");

// Pass coordinates of atom i at slot s.
template <int PREC>
__device__ __forceinline__ void v_store(const Dev& d, int s, int i, double x, double y, double z) {
    static_assert(PREC == 0, "MIXED lists are quad lists");
    reinterpret_cast<double4*>(d.vhi)[s] = make_double4(x, y, z, 0.0);
}

// ---------------------------------------------------------------- every step
// Pass coordinates, and the largest squared displacement since the rebuild under the step's parity
// (the other parity's slot is cleared for the next step).
template <int PREC> __global__ void k_v_pos(const Dev d, int k_local) {
    pdl_launch_dependents();
    pdl_wait();
    const int64_t step = *d.step_base + k_local;
    if (blockIdx.x == 0 && threadIdx.x == 0) d.vdmax[(step + 1) & 1] = 0u;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float dmax = 0.f;
    if (s < d.nslot) {
        const int np = d.npad, ns = d.nslot, i = d.vorder[s];
        const double x = d.x[i], y = d.x[np + i], z = d.x[2 * np + i];
        v_store<PREC>(d, s, i, x, y, z);
        const double ex = x - d.vxref[s], ey = y - d.vxref[ns + s], ez = z - d.vxref[2 * ns + s];
        dmax = (float)(ex * ex + ey * ey + ez * ez);
        if (!(dmax <= 3.0e38f)) dmax = 3.0e38f;  // non-finite positions force a rebuild
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0.f) atomicMax(d.vdmax + (step & 1), __float_as_uint(dmax));
}

// ---------------------------------------------------------------- rebuild
// One CTA per home cell (interior first), one warp per home octant; every staged atom closer than
// rcut + skin goes into the home atom's list. The home cell's atoms take consecutive list slots.
// The test runs in FP32 on the cell-centre offsets (errors ~1e-6 A); the rebuild trigger keeps a
// 1e-3 A margin, so a pair that can come within rcut before the next rebuild is always listed.
template <int PREC>
__global__ void __launch_bounds__(kCellThreads, 2) k_v_build(const Dev d, int cond, int k_local) {
    using V4 = typename Tr<PREC>::V4;
    using R = float;
    constexpr int TJ = kBuildTJ;
    __shared__ float4 spos[TJ];
    __shared__ int sidx[TJ];
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
    const CellGrid g = d.grid[d.cell_cl[c]];
    const V4* cp = reinterpret_cast<const V4*>(d.cpos);
    const int M = octant_box(d, c, g, s_src, s_cnt, s_pref);
    for (int k = threadIdx.x; k < hc; k += blockDim.x) s_len[k] = 0;
    if (threadIdx.x == 0) s_base = atomicAdd(d.vslot, hc);
    __syncthreads();
    const int base = s_base;
    for (int k = threadIdx.x; k < hc; k += blockDim.x) {
        const int a = d.cell_atoms[(size_t)c * kCellCap + k];
        d.vorder[base + k] = a;
        d.vslotof[a] = base + k;
        d.vrcount[base + k] = 0;
    }
    const R rl2 = (R)d.vrl2;
    const int nblk = oct_blocks(d, c), w = threadIdx.x >> 5;
    bool overflow = false;
    for (int blk = 0; blk < nblk; ++blk) {
        const OctWarp q = oct_warp(d, c, blk * 32);
        const int k_home = q.s0 + blk * 32 + q.is;  // the home atom's place in its cell
        const V4 pd = q.nb > 0 ? cp[(size_t)c * kCellCap + k_home] : V4{};
        const float4 pi = make_float4((float)pd.x, (float)pd.y, (float)pd.z, 0.f);
        const int me = q.nb > 0 ? d.cell_atoms[(size_t)c * kCellCap + k_home] : 0;
        int* list = d.vlist + (size_t)(base + k_home) * kVMax;
        for (int e0 = 0; e0 < M; e0 += TJ) {
            const int ne = min(TJ, M - e0);
            __syncthreads();
            for (int t = threadIdx.x; t < kBoxN; t += blockDim.x) {  // stage atoms, shifted to the home cell
                const int a = max(s_pref[t], e0), b = min(s_pref[t + 1], e0 + ne);
                const int dx = (t % kBox) / 2 - 1, dy = ((t / kBox) % kBox) / 2 - 1, dz = (t / (kBox * kBox)) / 2 - 1;
                const double sx = dx * g.h, sy = dy * g.h, sz = dz * g.h;
                for (int e = a; e < b; ++e) {
                    const int src = s_src[t] + (e - s_pref[t]);
                    const V4 p = cp[src];
                    spos[e - e0] = make_float4((float)(p.x + sx), (float)(p.y + sy), (float)(p.z + sz), 0.f);
                    sidx[e - e0] = d.cell_atoms[src];
                }
            }
            __syncthreads();
            oct_runs(s_pref, q.o, e0, ne, s_runs[w]);
            if (!q.act) continue;
            for (int run = 0; run < 25; ++run) {
                const int2 ab = s_runs[w][run];
                const int L = ab.y - ab.x, per = (L + q.J - 1) / q.J;
                const int lo = ab.x + min(L, q.jg * per), hi = ab.x + min(L, q.jg * per + per);
                for (int e = lo; e < hi; ++e) {
                    const float4 p = spos[e];
                    const R dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
                    const R r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (r2 < rl2 && sidx[e] > me) {  // half list: each pair once, at its lower atom
                        const int slot = atomicAdd(&s_len[k_home], 1);
                        if (slot < kVMax)
                            list[slot] = sidx[e];
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

// One warp per list: a bitonic sort of its entries by the key (j mod kVLanes, j); then the atoms
// are replaced by their slots and the end of every residue class is recorded.
__global__ void __launch_bounds__(kVThreads) k_v_sort(const Dev d, int cond, int k_local) {
    constexpr int HB = 32 - kVLog;  // the residue sits in the top kVLog bits of a key
    __shared__ uint32_t buf[kVThreads / 32][kVMax];
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * (kVThreads / 32) + w;
    if (s >= d.nslot) return;
    const int n = d.vcount[s];
    int P = 32;
    while (P < n) P <<= 1;
    uint32_t* b = buf[w];
    int* row = d.vlist + (size_t)s * kVMax;
    for (int e = lane; e < P; e += 32) {
        const uint32_t j = e < n ? (uint32_t)row[e] : 0u;
        b[e] = e < n ? ((j & (kVLanes - 1)) << HB) | (j >> kVLog) : 0xffffffffu;
    }
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
    const uint64_t ai = (uint64_t)(uint32_t)d.vorder[s];
    for (int e = lane; e < n; e += 32) {
        const uint32_t key = b[e];
        const uint32_t j = ((key & ((1u << HB) - 1)) << kVLog) | (key >> HB);
        const int sj = d.vslotof[j];
        row[e] = sj;
        // the partner's reverse list: (this atom, this entry's place), sorted in k_v_rsort by (atom mod
        // kVLanes, atom): the key's top kVLog bits hold the residue
        const int r = atomicAdd(d.vrcount + sj, 1);
        if (r < kVMax)
            d.vrev[(size_t)sj * kVMax + r] = (((ai & (kVLanes - 1)) << (64 - kVLog)) | ((ai >> kVLog) << 32)) |
                                             (uint32_t)((size_t)s * kVMax + e);
        else
            atomicOr(d.status, 4);
    }
    if (lane < kVLanes) {  // end of class `lane`: the first key of a higher class
        const uint32_t bound = (uint32_t)(lane + 1) << HB;
        int lo = 0, hi = n;
        if (lane == kVLanes - 1) lo = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (b[mid] < bound) lo = mid + 1; else hi = mid;
        }
        d.vsub[(size_t)s * kVLanes + lane] = lo;
    }
}

// One warp per slot: its reverse list (the entries of lower atoms that name it) sorted by (atom mod
// kVLanes, atom), a bitonic sort of the 64-bit keys; then the end of each residue class.
__global__ void __launch_bounds__(kVThreads) k_v_rsort(const Dev d, int cond, int k_local) {
    __shared__ uint64_t buf[kVThreads / 32][kVMax];
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * (kVThreads / 32) + w;
    if (s >= d.nslot) return;
    const int n = min(d.vrcount[s], kVMax);
    int P = 32;
    while (P < n) P <<= 1;
    uint64_t* b = buf[w];
    uint64_t* rv = d.vrev + (size_t)s * kVMax;
    for (int e = lane; e < P; e += 32) b[e] = e < n ? rv[e] : ~0ull;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = lane; e < P; e += 32) {
                const int f = e ^ j;
                if (f > e) {
                    const uint64_t x = b[e], y = b[f];
                    if ((x > y) == ((e & k) == 0)) {
                        b[e] = y;
                        b[f] = x;
                    }
                }
            }
            __syncwarp();
        }
    for (int e = lane; e < n; e += 32) rv[e] = b[e];
    if (lane < kVLanes) {  // end of class `lane`: the first key of a higher class
        const uint64_t bound = (uint64_t)(lane + 1) << (64 - kVLog);
        int lo = 0, hi = n;
        if (lane == kVLanes - 1) lo = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (b[mid] < bound) lo = mid + 1; else hi = mid;
        }
        d.vrsub[(size_t)s * kVLanes + lane] = lo;
    }
}

// Pass coordinates in the new slot order and the positions the next displacements are measured from.
template <int PREC> __global__ void k_v_commit(const Dev d, int cond, int k_local) {
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.nslot) return;
    const int np = d.npad, ns = d.nslot, i = d.vorder[s];
    const double x = d.x[i], y = d.x[np + i], z = d.x[2 * np + i];
    v_store<PREC>(d, s, i, x, y, z);
    d.vxref[s] = x;
    d.vxref[ns + s] = y;
    d.vxref[2 * ns + s] = z;
}

// ---------------------------------------------------------------- passes
// The sum of a double over the kVLanes threads of an atom, in a fixed tree (every thread gets it).
__device__ __forceinline__ double v_group_sum(double v) {
    const unsigned mask = ((1u << kVLanes) - 1u) << (threadIdx.x & 31 & ~(kVLanes - 1));
#pragma unroll
    for (int o = 1; o < kVLanes; o <<= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Half lists: atom i lists its partners j > i only. A pass computes each pair once; the term goes
// into i's own sum (registers) and is written at the entry's place for j. The gather kernels then
// add, for every atom, the terms of its reverse list in ascending order of the lower atom. Both
// orders are fixed by the positions alone, so the passes still do not depend on when the lists were
// built.

// One warp per atom, every MD step: the entries of its half list whose pair lies inside rcut now, in
// list order (a function of the positions alone), with a flag per list entry for the gathers.
__global__ void __launch_bounds__(kVThreads) k_v_compact(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= d.nslot) return;
    const double4* vp = reinterpret_cast<const double4*>(d.vhi);
    const double4 pi = vp[s];
    const double rc2 = d.pot.rcut2;
    const int n = d.vcount[s];
    const int* lst = d.vlist + (size_t)s * kVMax;
    int2* out = d.vcl + (size_t)s * kVMax;
    uint8_t* flag = d.vflag + (size_t)s * kVMax;
    int m = 0;
    for (int e0 = 0; e0 < n; e0 += 32) {
        const int e = e0 + lane;
        bool in = false;
        int q = 0;
        if (e < n) {
            q = lst[e];
            const double4 pj = vp[q];
            const double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            in = fma(dx, dx, fma(dy, dy, dz * dz)) < rc2;
            flag[e] = in ? 1 : 0;
        }
        const unsigned b = __ballot_sync(0xffffffffu, in);
        if (in) out[m + __popc(b & ((1u << lane) - 1u))] = make_int2(q, e);
        m += __popc(b);
    }
    if (lane == 0) d.vcn[s] = m;
}

// kVLanes threads per atom over its compacted entries (thread t takes entries t, t + kVLanes, ...),
// each pair inside rcut by construction. Each term goes into the atom's own sum and, for the
// partner, at the entry's place in the list.
template <int SPECIAL>
__global__ void __launch_bounds__(kVThreads) k_v_density(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = gt >> kVLog, t = gt & (kVLanes - 1);
    if (s >= d.nslot) return;  // whole atoms leave together
    const double4* vp = reinterpret_cast<const double4*>(d.vhi);
    const double4 pi = vp[s];
    const int n = d.vcn[s];
    const double shm = d.pot.shift ? d.pot.shm : 0.0;
    const int mexp = d.pot.m;
    const int2* cl = d.vcl + (size_t)s * kVMax;
    double* hb = d.hbuf + (size_t)s * kVMax;
    double racc = 0.0, tacc = 0.0;
    int cnt = 0, mine = 0;
#pragma unroll 4
    for (int k = t; k < n; k += kVLanes) {
        const int2 qe = cl[k];
        const double4 pj = vp[qe.x];
        const double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        double term;
        if (SPECIAL) {
            const double inv = inv_r2(r2);
            term = inv * inv * inv;
        } else {
            const double ir = inv_r(r2);
            term = rpow(ir * ir, ir, mexp);
        }
        tacc += term;
        hb[qe.y] = term - shm;
        ++mine;
        if (++cnt == kSpanV) {
            racc += tacc;
            tacc = 0.0;
            cnt = 0;
        }
    }
    racc += tacc;
    racc -= (double)mine * shm;
    racc = v_group_sum(racc);
    if (t == 0) d.rho_half[s] = racc;
}

// kVLanes threads per slot (thread t over the reverse-list entries of lower atoms a = t mod kVLanes,
// in ascending a), summed in a fixed tree and added to the atom's own sum; then the CTA's first
// threads finish its atoms, one each: rho and g.
__global__ void __launch_bounds__(kVThreads) k_v_dgather(const Dev d, int obs) {
    __shared__ double s_r[kVThreads / kVLanes];
    pdl_launch_dependents();
    pdl_wait();
    const int a = threadIdx.x >> kVLog, t = threadIdx.x & (kVLanes - 1);
    const int s = blockIdx.x * (kVThreads / kVLanes) + a;
    double r = 0.0;
    if (s < d.nslot) {
        const int beg = t ? d.vrsub[(size_t)s * kVLanes + t - 1] : 0, end = d.vrsub[(size_t)s * kVLanes + t];
        const uint64_t* rv = d.vrev + (size_t)s * kVMax;
#pragma unroll 4
        for (int k = beg; k < end; ++k) {  // entries outside rcut this step carry stale terms: skipped
            const uint32_t pos = (uint32_t)rv[k];
            if (d.vflag[pos]) r += d.hbuf[pos];
        }
    }
    r = v_group_sum(r);
    if (t == 0 && s < d.nslot) s_r[a] = d.rho_half[s] + r;
    __syncthreads();
    const int sl = blockIdx.x * (kVThreads / kVLanes) + threadIdx.x;  // one thread per atom of the CTA
    if (threadIdx.x >= kVThreads / kVLanes || sl >= d.nslot) return;
    const double rho = s_r[threadIdx.x] * d.pot.am;
    const int i = d.vorder[sl];
    d.rho[i] = rho;
    double4 p = reinterpret_cast<const double4*>(d.vhi)[sl];
    p.w = rho > 0.0 ? d.pot.B6 / sqrt(rho) : 0.0;
    reinterpret_cast<double4*>(d.vposg)[sl] = p;
    if (obs) d.eatom[2 * i] = -d.pot.eps * d.pot.c * sqrt(rho);
}

template <int SPECIAL, int ENERGY>
__global__ void __launch_bounds__(kVThreads) k_v_force(const Dev d) {
    pdl_launch_dependents();
    pdl_wait();
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = gt >> kVLog, t = gt & (kVLanes - 1);
    if (s >= d.nslot) return;  // whole atoms leave together
    const double4* vp = reinterpret_cast<const double4*>(d.vposg);
    const double4 pi = vp[s];
    const int n = d.vcn[s];
    const double A = d.pot.A9, shn = d.pot.shift ? d.pot.shn : 0.0;
    const int nexp = d.pot.n, mexp = d.pot.m;
    const int2* cl = d.vcl + (size_t)s * kVMax;
    double4* fb = d.fbuf + (size_t)s * kVMax;
    double fx = 0.0, fy = 0.0, fz = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, se = 0.0, ea = 0.0;
    int cnt = 0, mine = 0;
#pragma unroll 4
    for (int k = t; k < n; k += kVLanes) {
        const int2 qe = cl[k];
        const double4 pj = vp[qe.x];
        const double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double ir = inv_r(r2);
        const double inv = ir * ir;
        double coef, rn;
        if (SPECIAL) {
            const double inv2 = inv * inv, inv4 = inv2 * inv2;
            coef = inv4 * fma(A, inv * ir, -(pi.w + pj.w));
            rn = inv4 * ir;
        } else {
            rn = rpow(inv, ir, nexp);
            const double rm = rpow(inv, ir, mexp);
            coef = inv * (A * rn - (pi.w + pj.w) * rm);
        }
        const double ux = coef * dx, uy = coef * dy, uz = coef * dz;  // the force on i from j
        sx += ux;
        sy += uy;
        sz += uz;
        if (ENERGY) se += rn;
        fb[qe.y] = make_double4(ux, uy, uz, ENERGY ? rn - shn : 0.0);
        ++mine;
        if (++cnt == kSpanV) {
            fx += sx;
            fy += sy;
            fz += sz;
            sx = sy = sz = 0.0;
            if (ENERGY) {
                ea += se;
                se = 0.0;
            }
            cnt = 0;
        }
    }
    const double gx = v_group_sum(fx + sx), gy = v_group_sum(fy + sy), gz = v_group_sum(fz + sz);
    const double Ep = ENERGY ? v_group_sum(ea + se - (double)mine * shn) : 0.0;
    if (t == 0) d.fhalf[s] = make_double4(gx, gy, gz, Ep);
}

// kVLanes threads per slot: the force (and pair energy) terms of the reverse list, by residue class
// of the lower atom as in k_v_dgather, subtracted from (added to) the atom's own sums (Newton's third
// law); then the CTA's first threads do the per-atom work of the mode, one atom each: 0 forces;
// 1 forces and per-atom pair energies; 2 MD step (second half kick, per-atom observables if due,
// then the first half of the next step unless last or Berendsen).
template <int ENERGY>
__global__ void __launch_bounds__(kVThreads) k_v_fgather(const Dev d, int mode, int k_local, int last) {
    __shared__ double4 s_f[kVThreads / kVLanes];
    pdl_launch_dependents();
    pdl_wait();
    const int a = threadIdx.x >> kVLog, t = threadIdx.x & (kVLanes - 1);
    const int s = blockIdx.x * (kVThreads / kVLanes) + a;
    double ux = 0.0, uy = 0.0, uz = 0.0, ue = 0.0;
    if (s < d.nslot) {
        const int beg = t ? d.vrsub[(size_t)s * kVLanes + t - 1] : 0, end = d.vrsub[(size_t)s * kVLanes + t];
        const uint64_t* rv = d.vrev + (size_t)s * kVMax;
#pragma unroll 4
        for (int k = beg; k < end; ++k) {  // entries outside rcut this step carry stale terms: skipped
            const uint32_t pos = (uint32_t)rv[k];
            if (!d.vflag[pos]) continue;
            const double4 u = d.fbuf[pos];
            ux += u.x;
            uy += u.y;
            uz += u.z;
            if (ENERGY) ue += u.w;
        }
    }
    ux = v_group_sum(ux);
    uy = v_group_sum(uy);
    uz = v_group_sum(uz);
    if (ENERGY) ue = v_group_sum(ue);
    if (t == 0 && s < d.nslot) {
        const double4 h = d.fhalf[s];
        s_f[a] = make_double4(h.x - ux, h.y - uy, h.z - uz, h.w + ue);
    }
    __syncthreads();
    const int sl = blockIdx.x * (kVThreads / kVLanes) + threadIdx.x;  // one thread per atom of the CTA
    if (threadIdx.x >= kVThreads / kVLanes || sl >= d.nslot) return;
    const double4 F = s_f[threadIdx.x];
    const double Fx = F.x, Fy = F.y, Fz = F.z;
    const int i = d.vorder[sl];
    const int np = d.npad;
    double* fo = reinterpret_cast<double*>(d.f);
    fo[i] = Fx;
    fo[np + i] = Fy;
    fo[2 * np + i] = Fz;
    if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(d.status, 1);
    if (ENERGY) d.eatom[2 * i + 1] = F.w;
    if (mode != 2) return;
    const Run& r = *d.run;
    const int cl = d.cl_of_group[i >> 5];
    const double hs = d.hs[i];
    const double vx = fma(hs, Fx, d.v[i]);
    const double vy = fma(hs, Fy, d.v[np + i]);
    const double vz = fma(hs, Fz, d.v[2 * np + i]);
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
    if (!last) begin_step<0>(d, r, i, cl, i - d.poff[cl], *d.step_base + k_local + 1, Fx, Fy, Fz, k_local + 1);
}

// ---------------------------------------------------------------- launchers
// MIXED contexts run the quad lists (scmd_quads.cu).
cudaError_t launch_v_pos(const Dev& d, int k_local, cudaStream_t s) {
    if (d.prec == 1) return launch_q_pos(d, k_local, s);
    return launch_ex(k_v_pos<0>, (d.nslot + kVThreads - 1) / kVThreads, kVThreads, 0, 0, s, d, k_local);
}

cudaError_t launch_v_rebuild(const Dev& d, int cond, int k_local, cudaStream_t s) {
    if (d.prec == 1) return launch_q_rebuild(d, cond, k_local, s);
    const int wgrid = (d.nslot + kVThreads / 32 - 1) / (kVThreads / 32);  // one warp per slot
    cudaError_t e = launch_ex(k_v_build<0>, d.n_cells, kCellThreads, 0, 0, s, d, cond, k_local);
    if (e == cudaSuccess) e = launch_ex(k_v_sort, wgrid, kVThreads, 0, 0, s, d, cond, k_local);
    if (e == cudaSuccess) e = launch_ex(k_v_rsort, wgrid, kVThreads, 0, 0, s, d, cond, k_local);
    if (e != cudaSuccess) return e;
    return launch_ex(k_v_commit<0>, (d.nslot + kVThreads - 1) / kVThreads, kVThreads, 0, 0, s, d, cond, k_local);
}

static int v_pass_grid(const Dev& d) {
    return (int)(((int64_t)d.nslot * kVLanes + kVThreads - 1) / kVThreads);
}
static int v_gather_grid(const Dev& d) {  // kVLanes threads per slot
    return (d.nslot + kVThreads / kVLanes - 1) / (kVThreads / kVLanes);
}

cudaError_t launch_v_density(const Dev& d, int obs, cudaStream_t s, int k_local) {
    if (d.prec == 1) return launch_q_density(d, obs, k_local, s);
    cudaError_t e = launch_ex(k_v_compact, (d.nslot + kVThreads / 32 - 1) / (kVThreads / 32), kVThreads, 0, 0, s, d);
    if (e != cudaSuccess) return e;
    e = d.pot.special ? launch_ex(k_v_density<1>, v_pass_grid(d), kVThreads, 0, 0, s, d)
                      : launch_ex(k_v_density<0>, v_pass_grid(d), kVThreads, 0, 0, s, d);
    if (e != cudaSuccess) return e;
    return launch_ex(k_v_dgather, v_gather_grid(d), kVThreads, 0, 0, s, d, obs);
}

template <int ENERGY>
static cudaError_t v_force_e(const Dev& d, int mode, int k, int last, cudaStream_t s) {
    cudaError_t e = d.pot.special ? launch_ex(k_v_force<1, ENERGY>, v_pass_grid(d), kVThreads, 0, 0, s, d)
                                  : launch_ex(k_v_force<0, ENERGY>, v_pass_grid(d), kVThreads, 0, 0, s, d);
    if (e != cudaSuccess) return e;
    return launch_ex(k_v_fgather<ENERGY>, v_gather_grid(d), kVThreads, 0, 0, s, d, mode, k, last);
}

cudaError_t launch_v_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s) {
    if (d.prec == 1) return launch_q_force(d, mode, k_local, flags, s);
    const bool energy = (mode == 1) || (mode == 2 && (flags & 2));
    const int lst = flags & 1;
    return energy ? v_force_e<1>(d, mode, k_local, lst, s) : v_force_e<0>(d, mode, k_local, lst, s);
}

}  // namespace scmd
