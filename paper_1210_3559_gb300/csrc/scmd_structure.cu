// scmd_structure.cu -- structural observables of the clusters on the device (Sec. III): the
// pair-distance histogram of the central atoms, the mean squared displacement from a reference
// configuration, and common-neighbour analysis (CNA). Only small results leave the GPU (a
// histogram, one number or four counts per cluster, optionally one byte per atom).
//
// Distances that decide an integer (a histogram bin, a neighbour) are evaluated in FP64 with
// explicitly rounded operations in a fixed order -- dx = x_i - x_j per axis, r^2 = (dx dx + dy dy)
// + dz dz, r = sqrt(r^2), bin = r / width -- so the decision is the one plain IEEE arithmetic takes.
#include "scmd_internal.cuh"
#include "scmd_device.cuh"

namespace scmd {

namespace {

constexpr int kSThreads = 256;

__device__ __forceinline__ double r2_rn(double ax, double ay, double az, double bx, double by, double bz) {
    const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Centre of mass of cluster blockIdx.x into X (shared), summed in a fixed tree.
__device__ void block_com(const Dev& d, int p0, int n, double* X) {
    __shared__ double s[4][kSThreads];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    const int np = d.npad;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int i = p0 + t;
        const double m = d.mass[i];
        a[0] += m * d.x[i];
        a[1] += m * d.x[np + i];
        a[2] += m * d.x[2 * np + i];
        a[3] += m;
    }
    for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int w = kSThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) X[threadIdx.x] = s[3][0] > 0.0 ? s[threadIdx.x][0] / s[3][0] : 0.0;
    __syncthreads();
}

__device__ __forceinline__ bool within(const Dev& d, int i, const double* X, double r) {
    const int np = d.npad;
    return __dsqrt_rn(r2_rn(d.x[i], d.x[np + i], d.x[2 * np + i], X[0], X[1], X[2])) < r;
}

// ---------------------------------------------------------------- pair-distance histogram
// One CTA per cluster: its centre of mass and its core atoms (|x - X| < r_core), in any order.
__global__ void __launch_bounds__(kSThreads) k_rdf_core(const Dev d, StructBufs sb, double r_core) {
    __shared__ double X[3];
    __shared__ int s_n;
    pdl_launch_dependents();
    pdl_wait();
    const int b = blockIdx.x, p0 = d.poff[b], n = d.nreal[b];
    if (threadIdx.x == 0) s_n = 0;
    block_com(d, p0, n, X);
    for (int t = threadIdx.x; t < n; t += blockDim.x)
        if (within(d, p0 + t, X, r_core)) sb.core[p0 + atomicAdd(&s_n, 1)] = p0 + t;
    __syncthreads();
    if (threadIdx.x == 0) {
        sb.ncore[b] = s_n;
        for (int q = 0; q < 3; ++q) sb.com[3 * b + q] = X[q];
    }
}

// Y CTAs per cluster over its (core atom, other atom) pairs; integer counts, so the order of the
// additions does not matter.
__global__ void __launch_bounds__(kSThreads) k_rdf_hist(const Dev d, StructBufs sb, double width, int nbins, int Y) {
    extern __shared__ unsigned int h[];
    pdl_launch_dependents();
    pdl_wait();
    const int b = blockIdx.x / Y, y = blockIdx.x % Y;
    const int p0 = d.poff[b], n = d.nreal[b], nc = sb.ncore[b], np = d.npad;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) h[k] = 0u;
    __syncthreads();
    const int64_t total = (int64_t)nc * n;
    for (int64_t p = (int64_t)y * blockDim.x + threadIdx.x; p < total; p += (int64_t)Y * blockDim.x) {
        const int c = sb.core[p0 + (int)(p / n)], j = p0 + (int)(p % n);
        if (j == c) continue;
        const double r = __dsqrt_rn(r2_rn(d.x[c], d.x[np + c], d.x[2 * np + c], d.x[j], d.x[np + j], d.x[2 * np + j]));
        const double t = __ddiv_rn(r, width);
        if (t < (double)nbins) atomicAdd(&h[(int)t], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
        if (h[k]) atomicAdd(sb.hist + (size_t)b * nbins + k, (unsigned long long)h[k]);
}

// ---------------------------------------------------------------- mean squared displacement
__global__ void __launch_bounds__(kSThreads) k_msd_ref(const Dev d, StructBufs sb, double r_core) {
    __shared__ double X[3];
    pdl_launch_dependents();
    pdl_wait();
    const int b = blockIdx.x, p0 = d.poff[b], n = d.nreal[b], np = d.npad;
    block_com(d, p0, n, X);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int i = p0 + t;
        for (int q = 0; q < 3; ++q) sb.ref[q * np + i] = d.x[q * np + i];
        sb.sel[i] = (r_core <= 0.0 || within(d, i, X, r_core)) ? 1 : 0;
    }
    if (threadIdx.x < 3) sb.ref_com[3 * b + threadIdx.x] = X[threadIdx.x];
}

__global__ void __launch_bounds__(kSThreads) k_msd(const Dev d, StructBufs sb) {
    __shared__ double X[3];
    __shared__ double s[2][kSThreads];
    pdl_launch_dependents();
    pdl_wait();
    const int b = blockIdx.x, p0 = d.poff[b], n = d.nreal[b], np = d.npad;
    block_com(d, p0, n, X);
    const double* X0 = sb.ref_com + 3 * b;
    double acc = 0.0, cnt = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int i = p0 + t;
        if (!sb.sel[i]) continue;
        double d2 = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double e = __dsub_rn(__dsub_rn(d.x[q * np + i], X[q]), __dsub_rn(sb.ref[q * np + i], X0[q]));
            d2 = __dadd_rn(d2, __dmul_rn(e, e));
        }
        acc += d2;
        cnt += 1.0;
    }
    s[0][threadIdx.x] = acc;
    s[1][threadIdx.x] = cnt;
    __syncthreads();
    for (int w = kSThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sb.nsel[b] = (int)s[1][0];
        sb.msd[b] = s[1][0] > 0.0 ? s[0][0] / s[1][0] : 0.0;
    }
}

// ---------------------------------------------------------------- common-neighbour analysis
// One warp per 32-atom group (a group never straddles two clusters): lane l owns atom i; the warp
// walks its cluster in tiles of 32 atoms, each lane loading one as FP32 offsets from the cluster's
// first atom and the tile going round by shuffles. A pair that passes the FP32 test with a 0.01 A
// margin is decided in FP64. Neighbours are stored in ascending index, at most kNbCap of them; the
// count is exact.
__global__ void __launch_bounds__(kSThreads) k_cna_nb(const Dev d, StructBufs sb, double r_nb) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= d.ngroups) return;
    const int cl = d.cl_of_group[g], p0 = d.poff[cl], n = d.nreal[cl], np = d.npad;
    const int i = g * 32 + lane;
    const bool real = i - p0 < n;
    const double ox = d.x[p0], oy = d.x[np + p0], oz = d.x[2 * np + p0];
    const double xi = real ? d.x[i] : 0.0, yi = real ? d.x[np + i] : 0.0, zi = real ? d.x[2 * np + i] : 0.0;
    const float fx = (float)(xi - ox), fy = (float)(yi - oy), fz = (float)(zi - oz);
    const float lim = (float)((r_nb + 0.01) * (r_nb + 0.01));
    const double rn2 = __dmul_rn(r_nb, r_nb);
    int cnt = 0;
    int* out = sb.nb + (size_t)i * kNbCap;
    for (int t0 = 0; t0 < n; t0 += 32) {
        const int jl = p0 + t0 + lane;
        const bool jr = t0 + lane < n;
        const float jx = jr ? (float)(d.x[jl] - ox) : 3.0e38f;
        const float jy = jr ? (float)(d.x[np + jl] - oy) : 0.f;
        const float jz = jr ? (float)(d.x[2 * np + jl] - oz) : 0.f;
        for (int k = 0; k < 32; ++k) {
            const float ax = __shfl_sync(0xffffffffu, jx, k), ay = __shfl_sync(0xffffffffu, jy, k),
                        az = __shfl_sync(0xffffffffu, jz, k);
            const float ex = fx - ax, ey = fy - ay, ez = fz - az;
            const int j = p0 + t0 + k;
            if (real && j != i && ex * ex + ey * ey + ez * ez < lim &&
                r2_rn(xi, yi, zi, d.x[j], d.x[np + j], d.x[2 * np + j]) < rn2) {
                if (cnt < kNbCap) out[cnt] = j;
                ++cnt;
            }
        }
    }
    if (real) sb.nnb[i] = cnt;
}

// One warp per atom. With exactly 12 neighbours, lane k takes the bond to neighbour k: its row of
// the 12 x 12 adjacency among i's neighbours (bit m set when neighbour m is a neighbour of
// neighbour k) is the set of common neighbours of the bond. Then (k, b, l) = (common neighbours,
// bonds among them, bonds in the largest connected set of those bonds), from the rows by shuffles.
__global__ void __launch_bounds__(kSThreads) k_cna_class(const Dev d, StructBufs sb) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= d.npad) return;
    const int cl = d.cl_of_group[i >> 5];
    if (i - d.poff[cl] >= d.nreal[cl]) return;  // padding: the whole warp leaves
    const int n = sb.nnb[i];
    int cls = 0;
    bool capped = false;
    if (n == 12) {
        const int j = lane < 12 ? sb.nb[(size_t)i * kNbCap + lane] : 0;
        const int nj = lane < 12 ? sb.nnb[j] : 0;
        capped = __any_sync(0xffffffffu, nj > kNbCap);
        if (!capped) {
            unsigned row = 0u;
            for (int m = 0; m < 12; ++m) {
                const int target = __shfl_sync(0xffffffffu, j, m);
                if (lane < 12 && m != lane)
                    for (int e = 0; e < nj; ++e)
                        if (sb.nb[(size_t)j * kNbCap + e] == target) {
                            row |= 1u << m;
                            break;
                        }
            }
            unsigned rows[12];
#pragma unroll
            for (int m = 0; m < 12; ++m) rows[m] = __shfl_sync(0xffffffffu, row, m);
            const unsigned C = row;
            int bonds = 0;
#pragma unroll
            for (int m = 0; m < 12; ++m)
                if ((C >> m) & 1u) bonds += __popc(rows[m] & C);
            bonds /= 2;
            int chain = 0;
            unsigned left = C;
            while (left) {  // connected sets of the bond graph on C (at most 12 vertices)
                unsigned comp = left & (0u - left), grown = comp;
                do {
                    comp = grown;
#pragma unroll
                    for (int m = 0; m < 12; ++m)
                        if ((comp >> m) & 1u) grown |= rows[m] & C;
                } while (grown != comp);
                int e = 0;
#pragma unroll
                for (int m = 0; m < 12; ++m)
                    if ((comp >> m) & 1u) e += __popc(rows[m] & comp);
                chain = max(chain, e / 2);
                left &= ~comp;
            }
            const int kc = __popc(C);
            const bool s421 = lane < 12 && kc == 4 && bonds == 2 && chain == 1;
            const bool s422 = lane < 12 && kc == 4 && bonds == 2 && chain == 2;
            const bool s555 = lane < 12 && kc == 5 && bonds == 5 && chain == 5;
            const int n421 = __popc(__ballot_sync(0xffffffffu, s421));
            const int n422 = __popc(__ballot_sync(0xffffffffu, s422));
            const int n555 = __popc(__ballot_sync(0xffffffffu, s555));
            cls = n421 == 12 ? 1 : (n421 == 6 && n422 == 6) ? 2 : n555 == 12 ? 3 : 0;
        }
    }
    if (lane == 0) {
        sb.cls[i] = (int8_t)cls;
        atomicAdd(sb.counts + 4 * cl + cls, 1);
        if (capped) atomicAdd(sb.capped + cl, 1);
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_rdf(const Dev& d, const StructBufs& sb, double r_core, double width, int nbins, int Y,
                       cudaStream_t s) {
    cudaError_t e = launch_ex(k_rdf_core, d.B, kSThreads, 0, 0, s, d, sb, r_core);
    if (e != cudaSuccess) return e;
    return launch_ex(k_rdf_hist, d.B * Y, kSThreads, sizeof(unsigned int) * nbins, 0, s, d, sb, width, nbins, Y);
}

cudaError_t launch_msd_ref(const Dev& d, const StructBufs& sb, double r_core, cudaStream_t s) {
    return launch_ex(k_msd_ref, d.B, kSThreads, 0, 0, s, d, sb, r_core);
}

cudaError_t launch_msd(const Dev& d, const StructBufs& sb, cudaStream_t s) {
    return launch_ex(k_msd, d.B, kSThreads, 0, 0, s, d, sb);
}

cudaError_t launch_cna(const Dev& d, const StructBufs& sb, double r_nb, cudaStream_t s) {
    const int warps_per_cta = kSThreads / 32;
    cudaError_t e = launch_ex(k_cna_nb, (d.ngroups + warps_per_cta - 1) / warps_per_cta, kSThreads, 0, 0, s, d, sb,
                              r_nb);
    if (e != cudaSuccess) return e;
    return launch_ex(k_cna_class, (d.npad + warps_per_cta - 1) / warps_per_cta, kSThreads, 0, 0, s, d, sb);
}

}  // namespace scmd
