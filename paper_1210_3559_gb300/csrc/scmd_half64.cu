// scmd_half64.cu -- FP64 all-pairs passes that evaluate each pair once (Newton's third law).
//
// Both sweeps of the method (Sec. II, "Computational approach") are sums over pairs of terms
// symmetric in (i, j): the density term (a/r_ij)^m of Eq. 2 enters rho_i and rho_j, and the force
// term of the derivative of Eq. 1 enters F_i and, with the opposite sign, F_j. In FP64 the pair
// arithmetic runs on the FP64 pipe, which on this part has 1/64 of the FP32 rate, so evaluating
// each unordered pair once instead of twice nearly halves the passes' cost. (In MIXED precision
// the FP32 pipe is so fast that the extra shared-memory traffic of the second target would cost
// more than it saves; those passes stay on the ordered-pair kernels.)
//
// Work decomposition. A cluster of n atoms has T = ceil(n/32) i-tiles of 32 atoms and
// H = ceil(n/16) j half-tiles of 16 atoms. A work unit is (i-tile I, half-tile h) with h >= 2I:
//   * h in {2I, 2I+1} (the half-tiles inside tile I, "diagonal"): every ordered pair (i, j),
//     i in tile I, j in the half-tile, j != i, added to i only;
//   * h >= 2I+2: every unordered pair (i in tile I, j in half-tile h), added to i and to j.
// Each unordered pair of the cluster is thus visited exactly once. One warp takes a unit: lane l
// holds i = 32I + l; the 16 j atoms sit in shared memory; at step k = 0..15 lane l pairs with
// j = 16h + ((l + k) mod 16), so within each half of the warp the 16 lanes address 16 distinct
// j and add to their j-side sums (two copies per j, one per half-warp) without atomics.
// Each unit writes its i-side sums (32 atoms) and j-side sums (16 atoms) to its own slots; a
// second kernel adds an atom's slots in a fixed order (a fixed split over 8 warps, each taking
// every 8th of the atom's slots, then a fixed tree over the 8 partials) and finishes the pass
// (rho and g; or F and the integrator step). Results are deterministic run to run, so
// checkpoint/resume stays bitwise.
#include "scmd_device.cuh"

namespace scmd {
namespace {

constexpr int kHW = 4;  // warps (units) per CTA

// r^2 of a masked pair (self pair of a diagonal unit, or beyond the cutoff): finite, so that the
// Newton steps below stay finite, and far enough that every term underflows to 0.
constexpr double kMaskR2 = 1.0e300;

// FP64 reciprocal and reciprocal square root: the hardware's approximate values (MUFU) refined by two
// Newton-Raphson steps, each of which roughly doubles the number of correct bits, so the result is
// accurate to a few ulp. On the FP64 pipe this costs 4 (reciprocal) and 7 (reciprocal square root)
// multiply-adds; the pair passes' tolerances (1e-12 relative) need no correctly rounded result. The
// density pass uses the reciprocal (faster than the IEEE division); the force pass keeps the library's
// reciprocal square root, which measured faster than this one. Inputs must be finite and positive.
__device__ __forceinline__ double rcp_nr(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double h = 0.5 * x;
    y = y * fma(-h, y * y, 1.5);
    return y * fma(-h, y * y, 1.5);
}

// Unit of row X (i-tile X of the cluster) and half-tile h: (X, h) -> index within the cluster.
__device__ __forceinline__ int unit_index(int X, int h, int H) { return X * H - X * (X - 1) + (h - 2 * X); }

// The per-atom sum kernels: one CTA of kSW (16) warps per 32-atom group. An atom of tile X has K = (H - 2X) + X
// unit sums: term k < H - 2X is the i-side sum of unit (X, 2X + k), term k = H - 2X + J the j-side sum of
// unit (J, its half-tile), J < X. Warp w adds the terms k = w, w + kSW, ... of its lane's atom (every lane
// of a group has the same X, so the warps' loops are uniform); the kSW partials are then added in a fixed
// tree. Each dependent FP64 chain is thus ~K / kSW long instead of K (the FP64 add latency is 64 cycles).
constexpr int kSW = 16;

template <int NV>  // NV = 1: the .x component (density); 4: every component (force, pair energy)
__device__ __forceinline__ dbl4 unit_sums(const Dev& d, int la, int n, size_t ub, int warp) {
    const int H = (n + 15) >> 4, X = la >> 5, hA = la >> 4, ni = H - 2 * X, K = ni + X;
    const dbl4* pi = reinterpret_cast<const dbl4*>(d.h_pi);
    const dbl4* pj = reinterpret_cast<const dbl4*>(d.h_pj);
    const size_t r0 = ub + unit_index(X, 2 * X, H);
    dbl4 s = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int k = warp; k < K; k += kSW) {
        const dbl4* src = k < ni ? pi + (r0 + k) * 32 + (la & 31)
                                 : pj + (ub + unit_index(k - ni, hA, H)) * 16 + (la & 15);
        if (NV == 1) {  // density: compact doubles (the same slot index, 8 bytes per slot)
            s.x += k < ni ? reinterpret_cast<const double*>(d.h_pi)[(r0 + k) * 32 + (la & 31)]
                          : reinterpret_cast<const double*>(d.h_pj)[(ub + unit_index(k - ni, hA, H)) * 16 + (la & 15)];
        } else {
            const dbl4 t = *src;
            s.x += t.x;
            s.y += t.y;
            s.z += t.z;
            s.w += t.w;
        }
    }
    return s;
}

// Fixed-order tree over the kSW warp partials of lane t (red[w * 32 + t]).
__device__ __forceinline__ dbl4 tree_sw(const dbl4* red, int t) {
    dbl4 q[kSW];
#pragma unroll
    for (int w = 0; w < kSW; ++w) q[w] = red[w * 32 + t];
#pragma unroll
    for (int h = kSW / 2; h > 0; h >>= 1)
#pragma unroll
        for (int w = 0; w < h; ++w) q[w] = dbl4{q[w].x + q[w + h].x, q[w].y + q[w + h].y, q[w].z + q[w + h].z,
                                                 q[w].w + q[w + h].w};
    return q[0];
}

// ------------------------------------------------------------------ density
template <int SPECIAL, int CUT>
// These kernels do not trigger their dependents early (griddepcontrol.launch_dependents): they are
// launched with programmatic serialisation like the others, so the next kernel starts its launch when
// one of them completes. An early trigger let the next kernels (each triggering in turn) become
// resident and wait beside a pass that fills the FP64 pipe in one wave: the density pass took 132 µs
// per step at Ni~2000 instead of 62, the force pass 132 instead of 105.
__global__ void __launch_bounds__(32 * kHW) k_h_density(const Dev d) {
    __shared__ dbl4 tj[kHW][16];
    __shared__ double acc[kHW][32];  // [half-warp copy][16 j]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * kHW + warp;
    pdl_wait();  // positions come from the previous kernel
    if (u >= d.h_nunits) return;
    const int4 U = d.h_unit[u];  // (first i atom, first j atom, diagonal, cluster)
    const dbl4* mir = reinterpret_cast<const dbl4*>(d.mirror);
    const dbl4 pi = mir[U.x + lane];
    if (lane < 16) tj[warp][lane] = mir[U.y + lane];
    acc[warp][lane] = 0.0;
    __syncwarp();
    const double rc2 = d.pot.rcut2;
    const int mexp = d.pot.m, l16 = lane & 15, cbase = lane & 16;
    const bool diag = U.z != 0;
    double si = 0.0;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int jj = (l16 + k) & 15;
        const dbl4 p = tj[warp][jj];
        const double dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
        double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        if (CUT) r2 = (r2 < rc2) ? r2 : kMaskR2;
        if (diag && U.y + jj == U.x + lane) r2 = kMaskR2;
        double t;
        if (SPECIAL) {
            const double inv = rcp_nr(r2);
            t = inv * inv * inv;
        } else {
            const double ir = rsqrt_nr(r2);
            t = rpow(ir * ir, ir, mexp);
        }
        si += t;
        if (!diag) acc[warp][cbase + jj] += t;
        __syncwarp();
    }
    // the density pass stores its sums as compact doubles (a quarter of the force pass's slot)
    reinterpret_cast<double*>(d.h_pi)[(size_t)u * 32 + lane] = si;
    if (!diag && lane < 16) reinterpret_cast<double*>(d.h_pj)[(size_t)u * 16 + lane] = acc[warp][lane] + acc[warp][16 + lane];
}

// rho_i from the unit sums, then what the ordered-pair density pass's epilogue does: rho (FP64),
// g = B6 rho^-1/2 into posg, and the embedding-energy partials when observables are due.
__global__ void __launch_bounds__(32 * kSW) k_h_density_sum(const Dev d, int obs) {
    __shared__ dbl4 red[kSW * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = blockIdx.x;
    pdl_wait();
    const int i = g * 32 + lane, cl = d.cl_of_group[g];
    const int base = d.poff[cl], la = i - base, n = d.nreal[cl];
    const bool real = la < n;
    red[warp * 32 + lane] = real ? unit_sums<1>(d, la, n, (size_t)d.h_ubase[cl], warp) : dbl4{0.0, 0.0, 0.0, 0.0};
    __syncthreads();
    if (warp != 0) return;
    const double tot = tree_sw(red, lane).x;
    const double rho = tot * d.pot.am;
    if (real) {
        dbl4 p = reinterpret_cast<const dbl4*>(d.mirror)[i];
        p.w = rho > 0.0 ? d.pot.B6 / sqrt(rho) : 0.0;
        d.rho[i] = rho;
        reinterpret_cast<dbl4*>(d.posg)[i] = p;
    }
    if (obs) {
        double e = real ? -d.pot.eps * d.pot.c * sqrt(rho) : 0.0;
        e = warp_sum(e);
        if (lane == 0) d.part[(size_t)g * kObsFields + OF_EEMB] = e;
    }
}

// -------------------------------------------------------------------- force
template <int SPECIAL, int CUT, int ENERGY>
__global__ void __launch_bounds__(32 * kHW) k_h_force(const Dev d) {
    __shared__ dbl4 tj[kHW][16];
    __shared__ dbl4 acc[kHW][32];  // [half-warp copy][16 j]: (fx, fy, fz, sum r^-n)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * kHW + warp;
    pdl_wait();  // posg comes from the density pass
    if (u >= d.h_nunits) return;
    const int4 U = d.h_unit[u];
    const dbl4* pg = reinterpret_cast<const dbl4*>(d.posg);
    const dbl4 pi = pg[U.x + lane];
    if (lane < 16) tj[warp][lane] = pg[U.y + lane];
    acc[warp][lane] = dbl4{0.0, 0.0, 0.0, 0.0};
    __syncwarp();
    const double A = d.pot.A9, rc2 = d.pot.rcut2;
    const int nexp = d.pot.n, mexp = d.pot.m, l16 = lane & 15, cbase = lane & 16;
    const bool diag = U.z != 0;
    double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
#pragma unroll 2
    for (int k = 0; k < 16; ++k) {
        const int jj = (l16 + k) & 15;
        const dbl4 p = tj[warp][jj];
        const double dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
        double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        if (CUT) r2 = (r2 < rc2) ? r2 : kMaskR2;
        if (diag && U.y + jj == U.x + lane) r2 = kMaskR2;
        const double ir = inv_r(r2);  // (the Newton form measured slower than the library's here)
        const double inv = ir * ir;
        double coef, rn;
        if (SPECIAL) {
            const double inv2 = inv * inv, inv4 = inv2 * inv2;
            coef = inv4 * fma(A, inv * ir, -(pi.w + p.w));
            rn = inv4 * ir;
        } else {
            rn = rpow(inv, ir, nexp);
            const double rm = rpow(inv, ir, mexp);
            coef = inv * (A * rn - (pi.w + p.w) * rm);
        }
        fx = fma(coef, dx, fx);
        fy = fma(coef, dy, fy);
        fz = fma(coef, dz, fz);
        if (ENERGY) e += rn;
        if (!diag) {
            dbl4& a = acc[warp][cbase + jj];
            a.x = fma(-coef, dx, a.x);
            a.y = fma(-coef, dy, a.y);
            a.z = fma(-coef, dz, a.z);
            if (ENERGY) a.w += rn;
        }
        __syncwarp();
    }
    reinterpret_cast<dbl4*>(d.h_pi)[(size_t)u * 32 + lane] = dbl4{fx, fy, fz, e};
    if (!diag && lane < 16) {
        const dbl4 a = acc[warp][lane], b = acc[warp][16 + lane];
        reinterpret_cast<dbl4*>(d.h_pj)[(size_t)u * 16 + lane] = dbl4{a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w};
    }
}

// F_i and the pair-energy sum from the unit sums, then the force pass's epilogue (FP64): store F;
// mode 1: every observable partial at the current (x, v); mode 2: finish this MD step's half kick,
// record observables if due (flags bit 1), and start the next step unless it is the chunk's last
// (flags bit 0). The same arithmetic, in the same order, as the ordered-pair force pass.
__global__ void __launch_bounds__(32 * kSW) k_h_force_sum(const Dev d, int mode, int k_local, int flags) {
    __shared__ dbl4 red[kSW * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, group = blockIdx.x;
    pdl_wait();
    const int i = group * 32 + lane, cl = d.cl_of_group[group];
    const int base = d.poff[cl], la = i - base, n = d.nreal[cl];
    const bool real = la < n;
    red[warp * 32 + lane] = real ? unit_sums<4>(d, la, n, (size_t)d.h_ubase[cl], warp) : dbl4{0.0, 0.0, 0.0, 0.0};
    __syncthreads();
    if (warp != 0) return;
    const bool energy = mode == 1 || (mode == 2 && (flags & 2));
    const bool last = flags & 1;
    const dbl4 S = tree_sw(red, lane);
    const double Fx = S.x, Fy = S.y, Fz = S.z, Ep = S.w;
    const int np = d.npad;
    double* fo = reinterpret_cast<double*>(d.f);
    if (real) {
        fo[i] = Fx;
        fo[np + i] = Fy;
        fo[2 * np + i] = Fz;
        if (!(isfinite(Fx) && isfinite(Fy) && isfinite(Fz))) atomicOr(d.status, 1);
    }
    if (mode == 1) {
        const double mm = real ? d.mass[i] : 0.0;
        if (energy) {
            const double e = warp_sum(real ? Ep : 0.0);
            if (lane == 0) d.part[(size_t)group * kObsFields + OF_EPAIR] = e;
        }
        const double x = real ? d.x[i] : 0.0, y = real ? d.x[np + i] : 0.0, z = real ? d.x[2 * np + i] : 0.0;
        const double vx = real ? d.v[i] : 0.0, vy = real ? d.v[np + i] : 0.0, vz = real ? d.v[2 * np + i] : 0.0;
        obs_velocity_partials(d, group, real, mm, x, y, z, vx, vy, vz, lane);
        obs_position_partials(d, group, real, mm, x, y, z, lane);
        return;
    }
    if (mode != 2) return;
    const Run* rr = d.run;
    const int r_kind = rr->kind;
    const double vx0 = real ? d.v[i] : 0.0, vy0 = real ? d.v[np + i] : 0.0, vz0 = real ? d.v[2 * np + i] : 0.0;
    const double xx0 = real ? d.x[i] : 0.0, yy0 = real ? d.x[np + i] : 0.0, zz0 = real ? d.x[2 * np + i] : 0.0;
    const double hs = real ? d.hs[i] : 0.0, m = real ? d.mass[i] : 0.0;
    // velocities at the end of this step (second half kick)
    const double vx = fma(hs, Fx, vx0), vy = fma(hs, Fy, vy0), vz = fma(hs, Fz, vz0);
    if (energy) {  // observables are due at step + 1
        const double e = warp_sum(real ? Ep : 0.0);
        if (lane == 0) d.part[(size_t)group * kObsFields + OF_EPAIR] = e;
        obs_position_partials(d, group, real, m, xx0, yy0, zz0, lane);
        if (r_kind != 2) obs_velocity_partials(d, group, real, m, xx0, yy0, zz0, vx, vy, vz, lane);
    }
    if (r_kind == 2) {  // Berendsen: the rescale kernel finishes the step
        if (real) {
            d.v[i] = vx;
            d.v[np + i] = vy;
            d.v[2 * np + i] = vz;
        }
        const double ke2 = warp_sum(real ? m * (vx * vx + vy * vy + vz * vz) : 0.0);
        if (lane == 0) d.ke_grp[group] = ke2;
        return;
    }
    if (!real) return;
    if (last) {
        d.v[i] = vx;
        d.v[np + i] = vy;
        d.v[2 * np + i] = vz;
        return;
    }
    // next step (same arithmetic as begin_step): first half kick, then A O A or A A
    double ux = fma(hs, Fx, vx), uy = fma(hs, Fy, vy), uz = fma(hs, Fz, vz);
    double x, y, z;
    if (r_kind == 1) {
        const Run r = *rr;
        const int64_t s1 = *d.step_base + k_local + 1;
        double w[3];
        normals_f64(r.seed, (uint32_t)cl, s1, (uint32_t)la, w);
        const double sig = sqrt(r.noise_k * fmax(ramp_T(r, s1), 0.0) / m);
        const double nx = sig * w[0], ny = sig * w[1], nz = sig * w[2];
        x = fma(r.hk, ux, fma(r.h, nx, xx0));
        y = fma(r.hk, uy, fma(r.h, ny, yy0));
        z = fma(r.hk, uz, fma(r.h, nz, zz0));
        ux = fma(r.c1, ux, nx);
        uy = fma(r.c1, uy, ny);
        uz = fma(r.c1, uz, nz);
    } else {
        const double dt = rr->dt;
        x = fma(dt, ux, xx0);
        y = fma(dt, uy, yy0);
        z = fma(dt, uz, zz0);
    }
    store_mirror<0>(d, i, cl, x, y, z);
    d.v[i] = ux;
    d.v[np + i] = uy;
    d.v[2 * np + i] = uz;
    d.x[i] = x;
    d.x[np + i] = y;
    d.x[2 * np + i] = z;
    if (!(finite_bits(x) && finite_bits(y) && finite_bits(z) && finite_bits(ux) && finite_bits(uy) && finite_bits(uz)))
        atomicOr(d.status, 1);
}

template <int SP, int CUT>
cudaError_t density_h(const Dev& d, int obs, cudaStream_t s) {
    cudaError_t e = launch_ex(k_h_density<SP, CUT>, (d.h_nunits + kHW - 1) / kHW, 32 * kHW, 0, 0, s, d);
    if (e != cudaSuccess) return e;
    return launch_ex(k_h_density_sum, d.ngroups, 32 * kSW, 0, 0, s, d, obs);
}
template <int SP, int CUT, int EN>
cudaError_t force_h(const Dev& d, int mode, int k_local, int flags, cudaStream_t s) {
    cudaError_t e = launch_ex(k_h_force<SP, CUT, EN>, (d.h_nunits + kHW - 1) / kHW, 32 * kHW, 0, 0, s, d);
    if (e != cudaSuccess) return e;
    return launch_ex(k_h_force_sum, d.ngroups, 32 * kSW, 0, 0, s, d, mode, k_local, flags);
}

}  // namespace

cudaError_t launch_h_density(const Dev& d, int obs, cudaStream_t s) {
    const bool sp = d.pot.special != 0, cut = d.pot.rcut > 0.0;
    if (sp && !cut) return density_h<1, 0>(d, obs, s);
    if (sp && cut) return density_h<1, 1>(d, obs, s);
    if (!sp && !cut) return density_h<0, 0>(d, obs, s);
    return density_h<0, 1>(d, obs, s);
}

cudaError_t launch_h_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s) {
    const bool sp = d.pot.special != 0, cut = d.pot.rcut > 0.0;
    const bool en = (mode == 1) || (mode == 2 && (flags & 2));
    if (en) {
        if (sp && !cut) return force_h<1, 0, 1>(d, mode, k_local, flags, s);
        if (sp && cut) return force_h<1, 1, 1>(d, mode, k_local, flags, s);
        if (!sp && !cut) return force_h<0, 0, 1>(d, mode, k_local, flags, s);
        return force_h<0, 1, 1>(d, mode, k_local, flags, s);
    }
    if (sp && !cut) return force_h<1, 0, 0>(d, mode, k_local, flags, s);
    if (sp && cut) return force_h<1, 1, 0>(d, mode, k_local, flags, s);
    if (!sp && !cut) return force_h<0, 0, 0>(d, mode, k_local, flags, s);
    return force_h<0, 1, 0>(d, mode, k_local, flags, s);
}

}  // namespace scmd
