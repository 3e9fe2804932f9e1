// scmd_cells.cuh -- device helpers of the cell-list machinery shared by the cell-list pair
// passes (scmd_cells.cu) and the neighbour-list path (scmd_verlet.cu): the cell of a position,
// cell centres, the octant box around a home cell staged in shared memory, and the layout of one
// home octant per warp.
#pragma once
#include "scmd_device.cuh"

namespace scmd {


constexpr int kCellThreads = 256;
constexpr int kBox = 6, kBoxN = 216;  // the octant box of a home cell: 6 x 6 x 6 octants
template <int PREC> struct CellChunk;
template <> struct CellChunk<1> { static constexpr int TJ = 2304; };  // 36 KB of float4
template <> struct CellChunk<0> { static constexpr int TJ = 1024; };  // 32 KB of double4

// Cell index along one axis of a coordinate relative to the origin. fmin/fmax come before the
// conversion: far or non-finite coordinates land in a border cell.
__device__ __forceinline__ int cell_axis(double rel, const CellGrid& g) {
    return (int)fmin(fmax(floor((rel + g.E) * g.inv_h), 0.0), (double)(g.G - 1));
}
// Centre of cell k along one axis, relative to the origin (exact: h is a binary32 value).
__device__ __forceinline__ double cell_centre(int k, const CellGrid& g) { return -g.E + (k + 0.5) * g.h; }

// Neighbour-list path: a rebuild is due at local step k_local when some atom has moved more than
// skin / 2 since the last one (the largest squared displacement of that step, recorded by the anchor
// kernel under the step's parity).
__device__ __forceinline__ bool vlist_rebuild_due(const Dev& d, int k_local) {
    const int64_t step = *d.step_base + k_local;
    return __uint_as_float(d.vdmax[step & 1]) > d.vskin2h;
}

// The octant box of home cell c: the 27 cells around it, each split into its 2 x 2 x 2 octants of
// side h/2 >= rcut/2, form a 6 x 6 x 6 box of octants, numbered t = (Z * 6 + Y) * 6 + X. For each
// the source slot of its atoms (s_src) and the exclusive prefix of the counts in that order
// (s_pref[0..216]). Off-grid cells are empty. Every thread of the CTA calls this.
__device__ __forceinline__ int octant_box(const Dev& d, int c, const CellGrid& g, int* s_src, int* s_cnt,
                                          int* s_pref) {
    const int loc = c - g.off, cx = loc % g.G, cy = (loc / g.G) % g.G, cz = loc / (g.G * g.G);
    for (int t = threadIdx.x; t < kBoxN; t += blockDim.x) {
        const int X = t % kBox, Y = (t / kBox) % kBox, Z = t / (kBox * kBox);
        const int x = cx + X / 2 - 1, y = cy + Y / 2 - 1, z = cz + Z / 2 - 1;
        int n = 0, src = 0;
        if (x >= 0 && x < g.G && y >= 0 && y < g.G && z >= 0 && z < g.G) {
            const int nc = g.off + (z * g.G + y) * g.G + x, o = (X & 1) | ((Y & 1) << 1) | ((Z & 1) << 2);
            const int s0 = d.cell_oct[nc * 9 + o];
            n = d.cell_oct[nc * 9 + o + 1] - s0;
            src = nc * kCellCap + s0;
        }
        s_src[t] = src;
        s_cnt[t] = n;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 216 counts, 7 per lane
        const int lane = threadIdx.x;
        int v[7], sum = 0;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const int t = lane * 7 + q;
            v[q] = t < kBoxN ? s_cnt[t] : 0;
            sum += v[q];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        int run = incl - sum;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const int t = lane * 7 + q;
            if (t < kBoxN) s_pref[t] = run;
            run += v[q];
        }
        if (lane == 31) s_pref[kBoxN] = incl;
    }
    __syncthreads();
    return s_pref[kBoxN];
}

// Stage entries e0 .. e0 + ne - 1 of the octant box (one octant per thread), moved from their
// cell's centre to the home cell's centre by the exact (k - l) h.
template <class V4, class R>
__device__ __forceinline__ void gather_box(const V4* __restrict__ src, const int* s_src, const int* s_pref, R h,
                                           int e0, int ne, V4* spos) {
    for (int t = threadIdx.x; t < kBoxN; t += blockDim.x) {
        const int a = max(s_pref[t], e0), b = min(s_pref[t + 1], e0 + ne);
        if (a >= b) continue;
        const R sx = (R)((t % kBox) / 2 - 1) * h, sy = (R)(((t / kBox) % kBox) / 2 - 1) * h;
        const R sz = (R)((t / (kBox * kBox)) / 2 - 1) * h;
        const V4* from = src + s_src[t] - s_pref[t];
#pragma unroll 2
        for (int q = a; q < b; ++q) {
            V4 p = from[q];
            p.x += sx;
            p.y += sy;
            p.z += sz;
            spos[q - e0] = p;
        }
    }
}

// One home octant per warp: its atoms (cell slots s0 + r0 .. s0 + r0 + nb - 1), the staged place of
// its octant (for the self test) and the lane layout: nb i-slots times J = 32 / nb j-groups.
struct OctWarp {
    int o, s0, nb, J, is, jg, home_t;
    bool act;
};
__device__ __forceinline__ OctWarp oct_warp(const Dev& d, int c, int r0) {
    OctWarp q;
    const int lane = threadIdx.x & 31;
    q.o = threadIdx.x >> 5;
    q.s0 = d.cell_oct[c * 9 + q.o];
    q.nb = min(32, d.cell_oct[c * 9 + q.o + 1] - q.s0 - r0);
    q.J = q.nb > 0 ? 32 / q.nb : 1;
    q.is = q.nb > 0 ? lane % q.nb : 0;
    q.jg = q.nb > 0 ? lane / q.nb : 0;
    q.act = q.nb > 0 && q.jg < q.J;
    const int ox = q.o & 1, oy = (q.o >> 1) & 1, oz = q.o >> 2;
    q.home_t = ((2 + oz) * kBox + 2 + oy) * kBox + 2 + ox;
    return q;
}
// Blocks of 32 home atoms that the warp with the fullest octant needs (the same for every warp, so
// that the staging barriers line up).
__device__ __forceinline__ int oct_blocks(const Dev& d, int c) {
    int m = 0;
#pragma unroll
    for (int o = 0; o < 8; ++o) m = max(m, d.cell_oct[c * 9 + o + 1] - d.cell_oct[c * 9 + o]);
    return (m + 31) / 32;
}
// The 25 runs of the home octant's 5 x 5 x 5 neighbour octants (5 octants along x are adjacent in
// the staged order), clipped to the staged chunk [e0, e0 + ne): local [lo, hi) per run, written by
// the warp's lanes into its row of the run table.
__device__ __forceinline__ void oct_runs(const int* s_pref, int o, int e0, int ne, int2* runs) {
    const int lane = threadIdx.x & 31;
    if (lane < 25) {
        const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2, rz = lane / 5, ry = lane % 5;
        const int base = ((oz + rz) * kBox + oy + ry) * kBox + ox;
        const int a = max(s_pref[base], e0) - e0, b = min(s_pref[base + 5], e0 + ne) - e0;
        runs[lane] = make_int2(a, max(a, b));
    }
    __syncwarp();
}

}  // namespace scmd
