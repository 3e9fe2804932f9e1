// scmd_quads.cu -- MIXED neighbour lists kept per atom quad (the pair passes with a strict cutoff).
//
// Per-atom lists make every tested pair a gather of a random neighbour, and in FP32 those gathers,
// not the arithmetic, bound the passes. Here the unit is a quad: 4 consecutive slots of one cell,
// a compact group found by recursive bisection of the cell's atoms. Each quad keeps the list of
// the atoms, other than its own, within rcut + skin of one of its atoms at the last rebuild. A pass
// gives each quad a group of lanes, its 4 atoms in their registers: a lane gathers one listed atom
// at a time and tests it against all 4, so one gather serves 4 pairs. Per step:
//   k_q_pos    : every slot's offset from its quad's reference point, and the largest squared
//                displacement since the last rebuild (at a chunk's first step and with Berendsen;
//                otherwise the previous step's force pass, which moved the atoms, did this);
//   rebuild, when that displacement exceeds the trigger (the kernels exit at once otherwise):
//     the binning of the cell-list path (its sort is needless: the ranking below works from the binned
//                  order; its clearing too: k_q_order clears each cell's count once it has read it), then
//     k_q_scan   : the first slot of every cell (cells padded to whole quads), and the quad count;
//     k_q_order  : one CTA per cell: its atoms bisected into quads and placed in slots; per quad the
//                  reference point, the bounding box and the offsets;
//     k_q_list   : one warp per quad: the atoms of the 27 cells around it in reach of one of its
//                  atoms (the quads' boxes tested first);
//   k_q_density, k_q_force : kQLanes lanes per quad; per CTA of 8 quads, one warp then finishes the
//                32 atoms (the FP64 per-atom work on full warps).
// Coordinates: a quad's reference point C is its atoms' centroid rounded to a multiple of 2^-12 A,
// exact in FP32, so C_i - C_j is exact; an atom is stored as its FP32 offset o = x - C (|o| of a
// few A). A listed atom enters a pair as o_j - (C_i - C_j), rounded once, like the staged positions
// of the cell-list passes. The quad's own pairs are summed apart, where the self pair (r^2 = 0
// exactly) is masked; the lists hold no own atom, so their loop tests the cutoff alone.
// The sums run in list order, which depends on when the lists were built: unlike the FP64 lists,
// a resumed MIXED run agrees with an uninterrupted one to rounding, not bit for bit. Runs are
// deterministic: slots follow the cell order and lists the fixed order of the 27 cells.
#include <algorithm>
#include <climits>

#include "scmd_cells.cuh"

namespace scmd {

namespace {

constexpr int kQThreads = 256;  // the per-slot and list kernels (the list kernel: one warp per quad)
constexpr float kFar = kQuadFar;  // coordinate of an empty slot: outside every cutoff of every atom
// The quad build: one CTA of 128 threads per cell (a cell holds ~90 atoms at the fcc density), the grid
// capped at 16 CTAs per SM (larger batches stride). With 608 CTAs striding over the cells, a CTA that
// drew four occupied cells set the kernel's length (SM active cycles: 154 k at most against 88 k on
// average at Ni~50000).
constexpr int kQOrderThreads = 128;
constexpr int kQOrderGrid = 152 * 16;

// Quads by recursive bisection: a cell's n places (in atom-index order to start) form a segment; a
// segment of more than 4 places splits into a first part of 4 * floor(q / 2) places (q: its quads)
// and the rest, each part taking the atoms below / above the median along the segment's widest axis.
// Every part but a cell's last is then a whole number of quads, and the leaves are its quads.
// Place r's segment after lev splits:
__device__ __forceinline__ int2 kd_segment(int r, int n, int lev) {
    int b = 0, e = n;
    for (int l = 0; l < lev && e - b > 4; ++l) {
        const int n1 = 4 * (((e - b + 3) >> 2) >> 1);
        if (r < b + n1)
            e = b + n1;
        else
            b += n1;
    }
    return make_int2(b, e);
}
// A coordinate as an integer of the same order (a total order, NaN included, so ranks stay distinct),
// and back.
__device__ __forceinline__ int ord_key(float v) {
    const int b = __float_as_int(v);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// ---------------------------------------------------------------- every step
__global__ void __launch_bounds__(kQThreads) k_q_pos(const Dev d, int k_local) {
    pdl_launch_dependents();
    pdl_wait();
    const int64_t step = *d.step_base + k_local;
    if (blockIdx.x == 0 && threadIdx.x == 0) d.vdmax[(step + 1) & 1] = 0u;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float dmax = 0.f;
    const int i = s < 4 * *d.q_n ? d.vorder[s] : -1;
    if (i >= 0) {
        const int np = d.npad, ns = d.nslot;
        const double x = d.x[i], y = d.x[np + i], z = d.x[2 * np + i];
        const double* o = d.origin + 3 * d.cl_of_group[i >> 5];
        const float4 C = d.q_ref[s >> 2];
        reinterpret_cast<float4*>(d.vhi)[s] = make_float4((float)((x - o[0]) - (double)C.x),
                                                          (float)((y - o[1]) - (double)C.y),
                                                          (float)((z - o[2]) - (double)C.z), 0.f);
        const double ex = x - d.vxref[s], ey = y - d.vxref[ns + s], ez = z - d.vxref[2 * ns + s];
        dmax = (float)(ex * ex + ey * ey + ez * ez);
        if (!(dmax <= 3.0e38f)) dmax = 3.0e38f;  // non-finite positions force a rebuild
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0.f) atomicMax(d.vdmax + (step & 1), __float_as_uint(dmax));
}

// ---------------------------------------------------------------- rebuild
// One CTA: the first slot of every cell (its atoms padded to whole quads), in cell order.
__global__ void __launch_bounds__(1024) k_q_scan(const Dev d, int cond, int k_local) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < d.n_cells; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int v = c < d.n_cells ? (min(d.cell_count[c], kCellCap) + 3) & ~3 : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            int t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_warp[lane] = t;  // inclusive prefix over warps
        }
        __syncthreads();
        const int excl = s_carry + (w > 0 ? s_warp[w - 1] : 0) + x - v;
        if (c < d.n_cells) d.cell_base[c] = excl;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *d.q_n = s_carry >> 2;
        d.cell_base[d.n_cells] = s_carry;  // the end of the last cell
    }
}

// One CTA per cell: order its atoms into quads by recursive bisection, place them, and set up each of
// its quads.
__global__ void __launch_bounds__(kQOrderThreads) k_q_order(const Dev d, int cond, int k_local) {
    // per place, in the current order (two buffers): the 3 coordinates as order keys and the atom
    __shared__ int s_key[2][3][kCellCap];
    __shared__ int s_at[2][kCellCap];
    __shared__ int s_lo[kCellCap / 4][3], s_hi[kCellCap / 4][3];  // per segment (by its first quad)
    __shared__ int s_sorted[kCellCap];
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    for (int c = blockIdx.x; c < d.n_cells; c += gridDim.x) {  // a small grid: cheap when no rebuild is due
        __syncthreads();  // the previous cell's shared arrays are no longer read
        const int n = min(d.cell_count[c], kCellCap);
        if (n == 0) continue;
        const int cl = d.cell_cl[c];
        const float4* cp = reinterpret_cast<const float4*>(d.cposg);  // the binned order (no cell sort)
        const int* ca = d.cell_atoms + (size_t)c * kCellCap;
        for (int k = threadIdx.x; k < n; k += blockDim.x) s_sorted[k] = ca[k];  // (binned order)
        __syncthreads();
        // every thread has read the count: clear it for the next rebuild's binning (no clearing kernel;
        // the list kernel takes a cell's slot count from cell_base)
        if (threadIdx.x == 0) d.cell_count[c] = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {  // start: atom-index order
            const int a = s_sorted[k];
            int r = 0;
#pragma unroll 8
            for (int m = 0; m < n; ++m) r += s_sorted[m] < a;
            const float4 p = cp[(size_t)c * kCellCap + k];
            s_key[0][0][r] = ord_key(p.x);
            s_key[0][1][r] = ord_key(p.y);
            s_key[0][2][r] = ord_key(p.z);
            s_at[0][r] = a;
        }
        const int nq = (n + 3) >> 2;
        int cur = 0;
        for (int lev = 0; (1 << lev) < nq; ++lev, cur ^= 1) {
            __syncthreads();
            for (int r = threadIdx.x; r < n; r += blockDim.x) {  // the segments' extents (in key order)
                const int2 sg = kd_segment(r, n, lev);
                if (r == sg.x)
                    for (int q = 0; q < 3; ++q) s_lo[r >> 2][q] = INT_MAX, s_hi[r >> 2][q] = INT_MIN;
            }
            __syncthreads();
            for (int r0 = 0; r0 < n; r0 += blockDim.x) {  // (whole warps: the warp reductions below)
                const int r = r0 + threadIdx.x;
                const int2 sg = kd_segment(min(r, n - 1), n, lev);
                const bool act = r < n && sg.y - sg.x > 4;
                const int lead = __shfl_sync(0xffffffffu, sg.x, 0);
                if (__all_sync(0xffffffffu, act && sg.x == lead)) {  // one segment: reduce, then one atomic
                    for (int q = 0; q < 3; ++q) {
                        const int lo = __reduce_min_sync(0xffffffffu, s_key[cur][q][r]);
                        const int hi = __reduce_max_sync(0xffffffffu, s_key[cur][q][r]);
                        if ((threadIdx.x & 31) == 0) atomicMin(&s_lo[lead >> 2][q], lo), atomicMax(&s_hi[lead >> 2][q], hi);
                    }
                } else if (act) {
                    for (int q = 0; q < 3; ++q) {
                        atomicMin(&s_lo[sg.x >> 2][q], s_key[cur][q][r]);
                        atomicMax(&s_hi[sg.x >> 2][q], s_key[cur][q][r]);
                    }
                }
            }
            __syncthreads();
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                const int2 sg = kd_segment(r, n, lev);
                int to = r;
                if (sg.y - sg.x > 4) {
                    float w[3];
                    for (int q = 0; q < 3; ++q) w[q] = key_float(s_hi[sg.x >> 2][q]) - key_float(s_lo[sg.x >> 2][q]);
                    const int ax = (w[0] >= w[1] && w[0] >= w[2]) ? 0 : (w[1] >= w[2] ? 1 : 2);
                    const int* kk = s_key[cur][ax];
                    const int* at = s_at[cur];
                    const int v = kk[r], a = at[r];
                    int cnt = 0;
#pragma unroll 8
                    for (int m = sg.x; m < sg.y; ++m) cnt += kk[m] < v || (kk[m] == v && at[m] < a);
                    to = sg.x + cnt;
                }
                for (int q = 0; q < 3; ++q) s_key[cur ^ 1][q][to] = s_key[cur][q][r];
                s_at[cur ^ 1][to] = s_at[cur][r];
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) s_sorted[r] = s_at[cur][r];
        __syncthreads();
        const int base = d.cell_base[c], n4 = (n + 3) & ~3, ns = d.nslot, np = d.npad;
        for (int r = threadIdx.x; r < n4; r += blockDim.x) {
            const int a = r < n ? s_sorted[r] : -1;
            d.vorder[base + r] = a;
            if (a >= 0) d.vslotof[a] = base + r;
        }
        const double* o = d.origin + 3 * cl;
        for (int t = threadIdx.x; t < n4 / 4; t += blockDim.x) {
            const int Q = (base >> 2) + t;
            double rel[4][3], cen[3] = {0.0, 0.0, 0.0}, lo[3], hi[3];
            int cnt = 0;
            for (int u = 0; u < 4; ++u) {
                const int r = 4 * t + u;
                if (r >= n) break;
                const int a = s_sorted[r];
                for (int q = 0; q < 3; ++q) {
                    rel[u][q] = d.x[q * np + a] - o[q];
                    cen[q] += rel[u][q];
                    lo[q] = cnt == 0 ? rel[u][q] : fmin(lo[q], rel[u][q]);
                    hi[q] = cnt == 0 ? rel[u][q] : fmax(hi[q], rel[u][q]);
                }
                ++cnt;
            }
            float4 C;
            C.x = (float)(rint(cen[0] / cnt * 4096.0) * (1.0 / 4096.0));
            C.y = (float)(rint(cen[1] / cnt * 4096.0) * (1.0 / 4096.0));
            C.z = (float)(rint(cen[2] / cnt * 4096.0) * (1.0 / 4096.0));
            C.w = 0.f;
            d.q_ref[Q] = C;
            d.q_box[2 * Q] =
                make_float4(__double2float_rd(lo[0]), __double2float_rd(lo[1]), __double2float_rd(lo[2]), 0.f);
            d.q_box[2 * Q + 1] =
                make_float4(__double2float_ru(hi[0]), __double2float_ru(hi[1]), __double2float_ru(hi[2]), 0.f);
            d.q_cell[Q] = c;
            for (int u = 0; u < 4; ++u) {
                const int s = 4 * Q + u;
                float4 p = make_float4(kFar, kFar, kFar, 0.f);
                if (u < cnt) {
                    const int a = s_sorted[4 * t + u];
                    p = make_float4((float)(rel[u][0] - (double)C.x), (float)(rel[u][1] - (double)C.y),
                                    (float)(rel[u][2] - (double)C.z), 0.f);
                    d.vxref[s] = d.x[a];
                    d.vxref[ns + s] = d.x[np + a];
                    d.vxref[2 * ns + s] = d.x[2 * np + a];
                }
                reinterpret_cast<float4*>(d.vhi)[s] = p;
                reinterpret_cast<float4*>(d.vposg)[2 * s + 1] = C;  // the force pass's record: its quad's reference point
            }
        }
    }
}

// One warp per quad: the atoms of the 27 cells around its cell (fixed order; slot order within a
// cell) closer than rcut + skin to one of its atoms at the rebuild, its own atoms apart, appended in
// that order. One lane per candidate quad tests the bounding boxes; the quads whose boxes are in reach
// queue up (in order) in a per-warp buffer, and 8 at a time, one lane per atom, their atoms are tested
// against the 4 atoms of the warp's quad. So the exact tests run on full warps.
__global__ void __launch_bounds__(kQThreads) k_q_list(const Dev d, int cond, int k_local) {
    __shared__ int s_fifo[kQThreads / 32][64];  // quads whose boxes are in reach, not yet tested
    pdl_launch_dependents();
    pdl_wait();
    if (cond && !vlist_rebuild_due(d, k_local)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nq = *d.q_n;
    const unsigned lt = (1u << lane) - 1u;
    int* fifo = s_fifo[w];
    for (int Q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; Q < nq; Q += (gridDim.x * blockDim.x) >> 5) {
        const int c = d.q_cell[Q];
        const CellGrid g = d.grid[d.cell_cl[c]];
        const int loc = c - g.off, cx = loc % g.G, cy = (loc / g.G) % g.G, cz = loc / (g.G * g.G);
        const float4 lo = d.q_box[2 * Q], hi = d.q_box[2 * Q + 1];
        const float rl2 = (float)d.vrl2;
        const float4* vp = reinterpret_cast<const float4*>(d.vhi);
        float4 oi[4];
    #pragma unroll
        for (int a = 0; a < 4; ++a) oi[a] = vp[4 * Q + a];
        const float4 CI = d.q_ref[Q];
        int* out = d.q_list + (size_t)Q * kQMax;
        int n = 0, nf = 0;
        bool overflow = false;
        // the atoms of the first m (<= 8) queued quads: lane 4e + u takes atom u of quad e
        auto drain = [&](int m) {
            const int e = lane >> 2, sj = e < m ? 4 * fifo[e] + (lane & 3) : 0;
            bool in = false;
            if (e < m) {
                const float4 CJ = d.q_ref[sj >> 2], pj = vp[sj];  // an empty slot is far from all
                const float px = pj.x - (CI.x - CJ.x), py = pj.y - (CI.y - CJ.y), pz = pj.z - (CI.z - CJ.z);
    #pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float dx = oi[a].x - px, dy = oi[a].y - py, dz = oi[a].z - pz;
                    in |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rl2;
                }
            }
            const unsigned b = __ballot_sync(0xffffffffu, in);
            const int pos = n + __popc(b & lt);
            if (in) {
                if (pos < kQMax)
                    out[pos] = sj;
                else
                    overflow = true;
            }
            n += __popc(b);
            // the queue moves up by 8 (nf <= 39): every lane reads before any lane writes
            const int moved = lane + 8 < nf ? fifo[lane + 8] : 0;
            __syncwarp();
            if (lane + 8 < nf) fifo[lane] = moved;
            __syncwarp();
            nf = max(nf - 8, 0);
        };
        for (int nb = 0; nb < 27; ++nb) {
            const int x = cx + nb % 3 - 1, y = cy + (nb / 3) % 3 - 1, z = cz + nb / 9 - 1;
            if (x < 0 || x >= g.G || y < 0 || y >= g.G || z < 0 || z >= g.G) continue;
            const int c2 = g.off + (z * g.G + y) * g.G + x;
            const int q0 = d.cell_base[c2] >> 2, nq2 = (d.cell_base[c2 + 1] >> 2) - q0;
            for (int t0 = 0; t0 < nq2; t0 += 32) {
                const int J = q0 + t0 + lane;
                bool near = false;
                if (t0 + lane < nq2 && J != Q) {  // the quad's own pairs are summed apart from its list
                    const float4 l2 = d.q_box[2 * J], h2 = d.q_box[2 * J + 1];
                    const float ex = fmaxf(0.f, fmaxf(l2.x - hi.x, lo.x - h2.x));
                    const float ey = fmaxf(0.f, fmaxf(l2.y - hi.y, lo.y - h2.y));
                    const float ez = fmaxf(0.f, fmaxf(l2.z - hi.z, lo.z - h2.z));
                    near = ex * ex + ey * ey + ez * ez < rl2;
                }
                const unsigned b = __ballot_sync(0xffffffffu, near);
                if (near) fifo[nf + __popc(b & lt)] = J;
                nf += __popc(b);
                __syncwarp();
                while (nf >= 8) drain(8);
            }
        }
        if (nf > 0) drain(nf);
        if (lane == 0) d.q_count[Q] = min(n, kQMax);
        if (__any_sync(0xffffffffu, overflow) && lane == 0) atomicOr(d.status, 4);
        __syncwarp();  // the next quad reuses the queue
    }
}

// ---------------------------------------------------------------- passes
// A pass CTA takes 8 quads (32 slots) with kQLanes lanes per quad: lane seg of a quad's group takes
// list entries seg, seg + kQLanes, ... and pairs each with the 4 atoms of the quad, kept in registers.
// Then warp 0 finishes the 32 atoms with one lane each, so the FP64 per-atom work runs on full warps.
constexpr int kQLanes = 16;
constexpr int kQCta = 8;
constexpr int kQPassThreads = kQCta * kQLanes;
constexpr int kQPassMinCtas = 26 * 32 / kQPassThreads;  // resident CTAs per SM for >= 26 warps (the register cap)

// A listed atom pj of the quad with reference point CJ as an offset from the reference point CI of
// the lane's quad (the padding quad's slots land far from every atom and every empty slot).
__device__ __forceinline__ float4 q_shift(const float4& pj, const float4& CJ, const float4& CI) {
    return make_float4(pj.x - (CI.x - CJ.x), pj.y - (CI.y - CJ.y), pj.z - (CI.z - CJ.z), pj.w);
}
// Entry k of a list of n entries; past its end, a slot of the padding quad.
__device__ __forceinline__ int q_entry(const Dev& d, const int* L, int k, int n) { return k < n ? L[k] : 4 * d.nqmax; }
// Lanes 0..3 of a quad's group: atom seg of the quad, to be paired with its other three atoms before
// the list loop; the other lanes: far away.
__device__ __forceinline__ float4 q_self(const float4 oi[4], int seg) {
    float4 p = make_float4(-kFar, -kFar, -kFar, 0.f);
#pragma unroll
    for (int a = 0; a < 4; ++a)
        if (seg == a) p = oi[a];
    return p;
}
// Loop length of a warp: the longest list of its quads, rounded up to whole iterations (two entries per lane).
__device__ __forceinline__ int q_warp_len(int n) {
    const int m = __reduce_max_sync(0xffffffffu, n);
    return (m + 2 * kQLanes - 1) & ~(2 * kQLanes - 1);
}

// The 4 atoms of a quad (far away past the last quad) and the length of its list.
// REC: slots stored as 32-byte records (offset, then the quad's reference point: the force pass's array).
template <int REC>
__device__ __forceinline__ int q_own(const Dev& d, const float4* vp, int Q, int nq, float4 oi[4], float4& CI) {
    if (Q >= nq) {
#pragma unroll
        for (int a = 0; a < 4; ++a) oi[a] = make_float4(kFar, kFar, kFar, 0.f);
        CI = make_float4(0.f, 0.f, 0.f, 0.f);
        return 0;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) oi[a] = vp[(REC ? 2 : 1) * (4 * Q + a)];
    CI = d.q_ref[Q];
    return d.q_count[Q];
}

template <int SPECIAL, int SHIFT>
__global__ void __launch_bounds__(kQPassThreads, kQPassMinCtas) k_q_density(const Dev d, int obs, int k_local) {
    __shared__ f2sum s_sum[32];  // per slot: the density sum as double-float (FP64 only in warp 0's finish)
    __shared__ int s_nin[32];
    __shared__ float4 s_own[32];
    pdl_launch_dependents();
    pdl_wait();
    // in an MD step: clear the displacement record the force pass fills for the next step
    if (k_local >= 0 && blockIdx.x == 0 && threadIdx.x == 0) d.vdmax[(*d.step_base + k_local + 1) & 1] = 0u;
    const int lane = threadIdx.x & 31, g = threadIdx.x / kQLanes, seg = threadIdx.x % kQLanes;
    const int nq = *d.q_n, Q = blockIdx.x * kQCta + g;
    if (blockIdx.x * kQCta >= nq) return;  // the whole CTA is past the last quad
    const float4* vp = reinterpret_cast<const float4*>(d.vhi);
    float4 oi[4], CI;
    const int n = q_own<0>(d, vp, Q, nq, oi, CI);
    const int* L = d.q_list + (size_t)min(Q, nq - 1) * kQMax;
    const float rc2 = d.pot.rcut2f;  // (FP32 constants from the host: a conversion would run on the FP64 pipe)
    const int mexp = d.pot.m;
    float tacc[4] = {0.f, 0.f, 0.f, 0.f};
    int nin[4] = {0, 0, 0, 0};
#define SCMD_Q_DENSITY_PAIR(P, A, EXTRA)                                        \
    {                                                                           \
        const float dx = oi[A].x - P.x, dy = oi[A].y - P.y, dz = oi[A].z - P.z; \
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));                         \
        const bool in = r2 < rc2 EXTRA;                                         \
        r2 = in ? r2 : big<float>();                                            \
        if (SHIFT) nin[A] += in;                                                \
        if (SPECIAL) {                                                          \
            const float inv = inv_r2(r2);                                       \
            tacc[A] = fmaf(inv * inv, inv, tacc[A]);                            \
        } else {                                                                \
            const float ir = inv_r(r2);                                         \
            tacc[A] += rpow(ir * ir, ir, mexp);                                 \
        }                                                                       \
    }
    {  // the quad's own pairs (lanes 0..3 of the group); r2 > 0 also drops two empty slots of one quad
        const float4 p = q_self(oi, seg);
#pragma unroll
        for (int a = 0; a < 4; ++a) SCMD_Q_DENSITY_PAIR(p, a, && r2 > 0.f && a != seg)
    }
    // two listed atoms per lane and iteration; only the cutoff decides (no listed atom is one of the
    // quad's own)
    const int nw = q_warp_len(n);
    // the atoms are gathered one iteration ahead of their use, their list entries two ahead (past a
    // list's end: the padding quad)
    int s0 = q_entry(d, L, seg, n), s1 = q_entry(d, L, kQLanes + seg, n);
    float4 r0 = vp[s0], c0 = d.q_ref[s0 >> 2], r1 = vp[s1], c1 = d.q_ref[s1 >> 2];
    s0 = q_entry(d, L, 2 * kQLanes + seg, n);
    s1 = q_entry(d, L, 3 * kQLanes + seg, n);
    for (int k0 = 0; k0 < nw; k0 += 2 * kQLanes) {
        const float4 pp[2] = {q_shift(r0, c0, CI), q_shift(r1, c1, CI)};
        r0 = vp[s0];
        c0 = d.q_ref[s0 >> 2];
        r1 = vp[s1];
        c1 = d.q_ref[s1 >> 2];
        s0 = q_entry(d, L, k0 + 4 * kQLanes + seg, n);
        s1 = q_entry(d, L, k0 + 5 * kQLanes + seg, n);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 p = pp[h];
#pragma unroll
            for (int a = 0; a < 4; ++a) SCMD_Q_DENSITY_PAIR(p, a, )
        }
    }
#undef SCMD_Q_DENSITY_PAIR
#pragma unroll
    for (int a = 0; a < 4; ++a) {  // a fixed butterfly over the quad's lanes: each of them gets the sums
        // double-float (TwoSum) on the FP32 pipe: an FP64 butterfly here held the 1/64-rate FP64 pipe for
        // ~1/3 of the pass. TwoSum is exact, so both lanes of a pair compute the same sum.
        f2sum v = {tacc[a], 0.f};
        int m = nin[a];
#pragma unroll
        for (int o = 1; o < kQLanes; o <<= 1) {
            const f2sum u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
            v = f2_add(v, u);
            if (SHIFT) m += __shfl_xor_sync(0xffffffffu, m, o);
        }
        if (seg == a) {
            s_sum[4 * g + a] = v;
            if (SHIFT) s_nin[4 * g + a] = m;
            s_own[4 * g + a] = oi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32 || blockIdx.x * kQCta + (lane >> 2) >= nq) return;
    const int s = blockIdx.x * 4 * kQCta + lane, i = d.vorder[s];
    float4 pg = make_float4(kFar, kFar, kFar, 0.f);
    if (i >= 0) {
        const double t = (double)s_sum[lane].hi + (double)s_sum[lane].lo;
        const double rho = (SHIFT ? t - (double)s_nin[lane] * d.pot.shm : t) * d.pot.am;
        d.rho[i] = rho;
        const float rf = (float)rho;
        float y = rsqrt_approx(rf);
        y = y * (1.5f - 0.5f * rf * y * y);  // one Newton step
        const float4 me = s_own[lane];
        pg = make_float4(me.x, me.y, me.z, rho > 0.0 ? (float)d.pot.B6 * y : 0.0f);
        if (obs) d.eatom[2 * i] = -d.pot.eps * d.pot.c * sqrt(rho);
    }
    reinterpret_cast<float4*>(d.vposg)[2 * s] = pg;
}

// mode 0: forces; 1: forces and per-atom pair energies; 2: MD step (second half kick, per-atom
// observables if due, then the first half of the next step unless last or Berendsen).
template <int SPECIAL, int ENERGY>
__global__ void __launch_bounds__(kQPassThreads, kQPassMinCtas) k_q_force(const Dev d, int mode, int k_local, int last) {
    __shared__ float s_f[3][32];
    __shared__ double s_e[ENERGY ? 32 : 1];
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, g = threadIdx.x / kQLanes, seg = threadIdx.x % kQLanes;
    const int nq = *d.q_n, Q = blockIdx.x * kQCta + g;
    if (blockIdx.x * kQCta >= nq) return;  // the whole CTA is past the last quad
    const float4* vp = reinterpret_cast<const float4*>(d.vposg);
    float4 oi[4], CI;
    const int n = q_own<1>(d, vp, Q, nq, oi, CI);
    const int* L = d.q_list + (size_t)min(Q, nq - 1) * kQMax;
    const float A9 = d.pot.A9f, rc2 = d.pot.rcut2f;
    const int nexp = d.pot.n, mexp = d.pot.m;
    float fx[4] = {0.f, 0.f, 0.f, 0.f}, fy[4] = {0.f, 0.f, 0.f, 0.f}, fz[4] = {0.f, 0.f, 0.f, 0.f};
    float se[4] = {0.f, 0.f, 0.f, 0.f};
    int nin[4] = {0, 0, 0, 0};
#define SCMD_Q_FORCE_PAIR(P, A, EXTRA)                                          \
    {                                                                           \
        const float dx = oi[A].x - P.x, dy = oi[A].y - P.y, dz = oi[A].z - P.z; \
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));                         \
        const bool in = r2 < rc2 EXTRA;                                         \
        r2 = in ? r2 : big<float>();                                            \
        const float ir = inv_r(r2);                                             \
        const float inv = ir * ir;                                              \
        float coef, rn;                                                         \
        if (SPECIAL) {                                                          \
            const float inv2 = inv * inv, inv4 = inv2 * inv2;                   \
            coef = inv4 * fmaf(A9, inv * ir, -(oi[A].w + P.w));                 \
            rn = inv4 * ir;                                                     \
        } else {                                                                \
            rn = rpow(inv, ir, nexp);                                           \
            const float rm = rpow(inv, ir, mexp);                               \
            coef = inv * (A9 * rn - (oi[A].w + P.w) * rm);                      \
        }                                                                       \
        fx[A] = fmaf(coef, dx, fx[A]);                                          \
        fy[A] = fmaf(coef, dy, fy[A]);                                          \
        fz[A] = fmaf(coef, dz, fz[A]);                                          \
        if (ENERGY) {                                                           \
            se[A] += rn;                                                        \
            nin[A] += in;                                                       \
        }                                                                       \
    }
    {  // the quad's own pairs (lanes 0..3 of the group); r2 > 0 also drops two empty slots of one quad
        const float4 p = q_self(oi, seg);
#pragma unroll
        for (int a = 0; a < 4; ++a) SCMD_Q_FORCE_PAIR(p, a, && r2 > 0.f && a != seg)
    }
    // two listed atoms per lane and iteration; only the cutoff decides (no listed atom is one of the
    // quad's own)
    const int nw = q_warp_len(n);
    // the atoms are gathered one iteration ahead of their use, their list entries two ahead (past a
    // list's end: the padding quad)
    int s0 = q_entry(d, L, seg, n), s1 = q_entry(d, L, kQLanes + seg, n);
    // the slots are 32-byte records here: the listed atom and its quad's reference point in one sector
    float4 r0 = vp[2 * s0], c0 = vp[2 * s0 + 1], r1 = vp[2 * s1], c1 = vp[2 * s1 + 1];
    s0 = q_entry(d, L, 2 * kQLanes + seg, n);
    s1 = q_entry(d, L, 3 * kQLanes + seg, n);
    for (int k0 = 0; k0 < nw; k0 += 2 * kQLanes) {
        const float4 pp[2] = {q_shift(r0, c0, CI), q_shift(r1, c1, CI)};
        r0 = vp[2 * s0];
        c0 = vp[2 * s0 + 1];
        r1 = vp[2 * s1];
        c1 = vp[2 * s1 + 1];
        s0 = q_entry(d, L, k0 + 4 * kQLanes + seg, n);
        s1 = q_entry(d, L, k0 + 5 * kQLanes + seg, n);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 p = pp[h];
#pragma unroll
            for (int a = 0; a < 4; ++a) SCMD_Q_FORCE_PAIR(p, a, )
        }
    }
#undef SCMD_Q_FORCE_PAIR
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float x = fx[a], y = fy[a], z = fz[a];
        double e = ENERGY ? (double)se[a] : 0.0;
        int m = nin[a];
#pragma unroll
        for (int o = 1; o < kQLanes; o <<= 1) {  // a fixed butterfly over the quad's lanes
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
            if (ENERGY) {
                e += __shfl_xor_sync(0xffffffffu, e, o);
                m += __shfl_xor_sync(0xffffffffu, m, o);
            }
        }
        if (seg == a) {
            s_f[0][4 * g + a] = x;
            s_f[1][4 * g + a] = y;
            s_f[2][4 * g + a] = z;
            if (ENERGY) s_e[4 * g + a] = e - (d.pot.shift ? (double)m * d.pot.shn : 0.0);
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    // warp 0: one lane per slot of the CTA's 8 quads
    const int sl = blockIdx.x * 4 * kQCta + lane;
    const int i = blockIdx.x * kQCta + (lane >> 2) < nq ? d.vorder[sl] : -1;
    const Run& r = *d.run;
    // in an MD step (not the chunk's last, not Berendsen) this kernel starts the next step, so it also
    // does the position kernel's work for it: the slot's offset and the displacement since the rebuild
    const bool next = mode == 2 && !last && r.kind != 2;
    float dmax = 0.f;
    if (i >= 0) {
        const float Fx = s_f[0][lane], Fy = s_f[1][lane], Fz = s_f[2][lane];
        const int np = d.npad;
        float* fo = reinterpret_cast<float*>(d.f);
        fo[i] = Fx;
        fo[np + i] = Fy;
        fo[2 * np + i] = Fz;
        if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(d.status, 1);
        if (ENERGY) d.eatom[2 * i + 1] = s_e[lane];
        if (mode == 2) {
            const int cl = d.cl_of_group[i >> 5];
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
                if (!last) {
                    begin_step<1>(d, r, i, cl, i - d.poff[cl], *d.step_base + k_local + 1, (double)Fx, (double)Fy,
                                  (double)Fz, k_local + 1);
                    const double x = d.x[i], y = d.x[np + i], z = d.x[2 * np + i];
                    const double* o = d.origin + 3 * cl;
                    const float4 C = d.q_ref[sl >> 2];
                    reinterpret_cast<float4*>(d.vhi)[sl] =
                        make_float4((float)((x - o[0]) - (double)C.x), (float)((y - o[1]) - (double)C.y),
                                    (float)((z - o[2]) - (double)C.z), 0.f);
                    const int ns = d.nslot;
                    const double ex = x - d.vxref[sl], ey = y - d.vxref[ns + sl], ez = z - d.vxref[2 * ns + sl];
                    dmax = (float)(ex * ex + ey * ey + ez * ez);
                    if (!(dmax <= 3.0e38f)) dmax = 3.0e38f;  // non-finite positions force a rebuild
                }
            }
        }
    }
    if (next) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (lane == 0 && dmax > 0.f)
            atomicMax(d.vdmax + ((*d.step_base + k_local + 1) & 1), __float_as_uint(dmax));
    }
}

int q_pass_grid(const Dev& d) { return (d.nqmax + kQCta - 1) / kQCta; }

template <int SHIFT> cudaError_t q_density_s(const Dev& d, int obs, int k_local, cudaStream_t s) {
    return d.pot.special ? launch_ex(k_q_density<1, SHIFT>, q_pass_grid(d), kQPassThreads, 0, 0, s, d, obs, k_local)
                         : launch_ex(k_q_density<0, SHIFT>, q_pass_grid(d), kQPassThreads, 0, 0, s, d, obs, k_local);
}

template <int ENERGY> cudaError_t q_force_e(const Dev& d, int mode, int k, int last, cudaStream_t s) {
    return d.pot.special ? launch_ex(k_q_force<1, ENERGY>, q_pass_grid(d), kQPassThreads, 0, 0, s, d, mode, k, last)
                         : launch_ex(k_q_force<0, ENERGY>, q_pass_grid(d), kQPassThreads, 0, 0, s, d, mode, k, last);
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_q_pos(const Dev& d, int k_local, cudaStream_t s) {
    return launch_ex(k_q_pos, (d.nslot + kQThreads - 1) / kQThreads, kQThreads, 0, 0, s, d, k_local);
}

cudaError_t launch_q_rebuild(const Dev& d, int cond, int k_local, cudaStream_t s) {
    cudaError_t e = launch_ex(k_q_scan, 1, 1024, 0, 0, s, d, cond, k_local);
    if (e != cudaSuccess) return e;
    // small grids: most steps these kernels only check that no rebuild is due
    e = launch_ex(k_q_order, std::min(d.n_cells, kQOrderGrid), kQOrderThreads, 0, 0, s, d, cond, k_local);
    if (e != cudaSuccess) return e;
    return launch_ex(k_q_list, std::min(q_pass_grid(d), 608), kQThreads, 0, 0, s, d, cond, k_local);
}

cudaError_t launch_q_density(const Dev& d, int obs, int k_local, cudaStream_t s) {
    return d.pot.shift ? q_density_s<1>(d, obs, k_local, s) : q_density_s<0>(d, obs, k_local, s);
}

cudaError_t launch_q_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s) {
    const bool energy = (mode == 1) || (mode == 2 && (flags & 2));
    const int lst = flags & 1;
    return energy ? q_force_e<1>(d, mode, k_local, lst, s) : q_force_e<0>(d, mode, k_local, lst, s);
}

}  // namespace scmd
