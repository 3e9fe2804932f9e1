// scmd_device.cuh -- device helpers shared by the pair-pass kernels of libscmd: precision
// traits, MUFU wrappers, Philox4x32-10 and Box-Muller, the velocity-Verlet / BAOAB step of one
// atom, observable partials, double-float sums, programmatic-dependent-launch and
// thread-block-cluster barrier wrappers, cp.async, and the launch helper.
#pragma once
#include <cooperative_groups.h>

#include <cmath>
#include <cstdint>

#include "scmd_internal.cuh"

namespace cg = cooperative_groups;

namespace scmd {


struct __align__(32) dbl4 {
    double x, y, z, w;
};

template <int PREC> struct Tr;
template <> struct Tr<1> {
    using R = float;
    using V4 = float4;
};
template <> struct Tr<0> {
    using R = double;
    using V4 = dbl4;
};

// PTX approximate reciprocal / reciprocal square root (one MUFU op each).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float inv_r2(float r2) { return rcp_approx(r2); }
__device__ __forceinline__ double inv_r2(double r2) { return 1.0 / r2; }
__device__ __forceinline__ float inv_r(float r2) { return rsqrt_approx(r2); }
__device__ __forceinline__ double inv_r(double r2) { return rsqrt(r2); }

template <class R> __device__ __forceinline__ R ipow(R b, int e) {
    R r = R(1);
    for (int k = 0; k < e; ++k) r *= b;
    return r;
}
// r^-k from ir = r^-1 and inv = r^-2 (runtime exponent)
template <class R> __device__ __forceinline__ R rpow(R inv, R ir, int k) {
    R p = ipow(inv, k >> 1);
    return (k & 1) ? p * ir : p;
}

template <class R> __device__ __forceinline__ R big();
template <> __device__ __forceinline__ float big<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double big<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ Philox / normals
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
        const uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Three standard normals for (atom, cluster, step): Box-Muller on (w0,w1), (w2,w3).
__device__ __forceinline__ void normals_f32(uint64_t seed, uint32_t cl, int64_t step, uint32_t atom, float z[3]) {
    uint32_t c[4] = {atom, cl, (uint32_t)((uint64_t)step & 0xffffffffu), (uint32_t)((uint64_t)step >> 32)};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const float s32 = 2.3283064365386963e-10f;  // 2^-32
    const float u1 = fmaf((float)c[0], s32, s32), u2 = fmaf((float)c[1], s32, s32);
    const float u3 = fmaf((float)c[2], s32, s32), u4 = fmaf((float)c[3], s32, s32);
    const float r1 = sqrtf(-2.0f * logf(u1)), r2 = sqrtf(-2.0f * logf(u3));
    float s1, c1, s2, c2;
    sincospif(2.0f * u2, &s1, &c1);
    sincospif(2.0f * u4, &s2, &c2);
    z[0] = r1 * c1;
    z[1] = r1 * s1;
    z[2] = r2 * c2;
}
__device__ __forceinline__ void normals_f64(uint64_t seed, uint32_t cl, int64_t step, uint32_t atom, double z[3]) {
    uint32_t c[4] = {atom, cl, (uint32_t)((uint64_t)step & 0xffffffffu), (uint32_t)((uint64_t)step >> 32)};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const double s32 = 2.3283064365386963e-10;
    const double u1 = ((double)c[0] + 1.0) * s32, u2 = ((double)c[1] + 1.0) * s32;
    const double u3 = ((double)c[2] + 1.0) * s32, u4 = ((double)c[3] + 1.0) * s32;
    const double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
    double s1, c1, s2, c2;
    sincospi(2.0 * u2, &s1, &c1);
    sincospi(2.0 * u4, &s2, &c2);
    z[0] = r1 * c1;
    z[1] = r1 * s1;
    z[2] = r2 * c2;
}

// ------------------------------------------------------------------ helpers
// Exponent-field test on the integer pipe (IEEE double finite iff exponent != all ones).
__device__ __forceinline__ bool finite_bits(double v) {
    return (__double_as_longlong(v) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

__device__ __forceinline__ double ramp_T(const Run& r, int64_t step) {
    return r.T0 + r.dT * (double)(step - r.step0);
}

// MIXED: float(x - o) with the cluster's fixed origin o. FP64: the position itself.
template <int PREC> __device__ __forceinline__ void store_mirror(const Dev& d, int i, int cl, double x, double y, double z) {
    using V4 = typename Tr<PREC>::V4;
    V4 p;
    if (PREC == 1) {
        const double* o = d.origin + 3 * cl;
        p.x = (float)(x - o[0]);
        p.y = (float)(y - o[1]);
        p.z = (float)(z - o[2]);
    } else {
        p.x = x;
        p.y = y;
        p.z = z;
    }
    p.w = 0;
    reinterpret_cast<V4*>(d.mirror)[i] = p;
}

template <int PREC> __device__ __forceinline__ void load_force(const Dev& d, int i, double& fx, double& fy, double& fz) {
    using R = typename Tr<PREC>::R;
    const R* f = reinterpret_cast<const R*>(d.f);
    fx = (double)f[i];
    fy = (double)f[d.npad + i];
    fz = (double)f[2 * d.npad + i];
}

// Start of a step for one atom from (x, v, F): B, then A O A (Langevin) or A A (NVE, Berendsen).
// Per-atom factors h conv / m and the Langevin noise scale come precomputed (k_prepare), so the
// FP64 work here is multiply-adds only. With u the velocity after B and n the O-step noise, BAOAB
// gives v' = c1 u + n and x' = x + h u + h v' = x + h n + h (1 + c1) u, evaluated in that form
// (shared with the force-pass epilogue, so that a step starting a chunk rounds like any other).
template <int PREC>
__device__ __forceinline__ void begin_step(const Dev& d, const Run& r, int i, int cl, int atom, int64_t step,
                                           double fx, double fy, double fz, int noise_slot) {
    const int np = d.npad;
    const double hs = d.hs[i];
    double ux = fma(hs, fx, d.v[i]), uy = fma(hs, fy, d.v[np + i]), uz = fma(hs, fz, d.v[2 * np + i]);
    const double x0 = d.x[i], y0 = d.x[np + i], z0 = d.x[2 * np + i];
    double x, y, z;
    if (r.kind == 1) {
        double nx, ny, nz;
        if (PREC == 1) {
            float4 zz;
            if (noise_slot >= 0) {
                zz = d.noise[(size_t)noise_slot * np + i];  // already times sqrt(T(step))
            } else {
                float w[3];
                normals_f32(r.seed, (uint32_t)cl, step, (uint32_t)atom, w);
                const float sT = sqrtf((float)fmax(ramp_T(r, step), 0.0));
                zz = make_float4(w[0] * sT, w[1] * sT, w[2] * sT, 0.f);
            }
            const float sg = d.sig0[i];
            nx = (double)(sg * zz.x);
            ny = (double)(sg * zz.y);
            nz = (double)(sg * zz.z);
        } else {
            double w[3];
            normals_f64(r.seed, (uint32_t)cl, step, (uint32_t)atom, w);
            const double sig = sqrt(r.noise_k * fmax(ramp_T(r, step), 0.0) / d.mass[i]);
            nx = sig * w[0];
            ny = sig * w[1];
            nz = sig * w[2];
        }
        x = fma(r.hk, ux, fma(r.h, nx, x0));
        y = fma(r.hk, uy, fma(r.h, ny, y0));
        z = fma(r.hk, uz, fma(r.h, nz, z0));
        ux = fma(r.c1, ux, nx);
        uy = fma(r.c1, uy, ny);
        uz = fma(r.c1, uz, nz);
    } else {
        x = fma(r.dt, ux, x0);
        y = fma(r.dt, uy, y0);
        z = fma(r.dt, uz, z0);
    }
    d.v[i] = ux;
    d.v[np + i] = uy;
    d.v[2 * np + i] = uz;
    d.x[i] = x;
    d.x[np + i] = y;
    d.x[2 * np + i] = z;
    if (!(finite_bits(x) && finite_bits(y) && finite_bits(z) && finite_bits(ux) && finite_bits(uy) && finite_bits(uz)))
        atomicOr(d.status, 1);
    store_mirror<PREC>(d, i, cl, x, y, z);
}

// Velocity-dependent observable partials of one warp-group (lane values -> lane 0 writes).
__device__ __forceinline__ void obs_velocity_partials(const Dev& d, int group, bool real, double m, double x, double y,
                                                      double z, double vx, double vy, double vz, int lane) {
    double ke2 = real ? m * (vx * vx + vy * vy + vz * vz) : 0.0;
    double px = real ? m * vx : 0.0, py = real ? m * vy : 0.0, pz = real ? m * vz : 0.0;
    double lx = real ? m * (y * vz - z * vy) : 0.0;
    double ly = real ? m * (z * vx - x * vz) : 0.0;
    double lz = real ? m * (x * vy - y * vx) : 0.0;
    ke2 = warp_sum(ke2);
    px = warp_sum(px);
    py = warp_sum(py);
    pz = warp_sum(pz);
    lx = warp_sum(lx);
    ly = warp_sum(ly);
    lz = warp_sum(lz);
    if (lane == 0) {
        double* p = d.part + (size_t)group * kObsFields;
        p[OF_KE2] = ke2;
        p[OF_P] = px;
        p[OF_P + 1] = py;
        p[OF_P + 2] = pz;
        p[OF_L] = lx;
        p[OF_L + 1] = ly;
        p[OF_L + 2] = lz;
    }
}
__device__ __forceinline__ void obs_position_partials(const Dev& d, int group, bool real, double m, double x, double y,
                                                      double z, int lane) {
    double mx = real ? m * x : 0.0, my = real ? m * y : 0.0, mz = real ? m * z : 0.0, mm = real ? m : 0.0;
    mx = warp_sum(mx);
    my = warp_sum(my);
    mz = warp_sum(mz);
    mm = warp_sum(mm);
    if (lane == 0) {
        double* p = d.part + (size_t)group * kObsFields;
        p[OF_MX] = mx;
        p[OF_MX + 1] = my;
        p[OF_MX + 2] = mz;
        p[OF_MASS] = mm;
    }
}

// ------------------------------------------------------- double-float sums
// An unevaluated sum hi + lo of two FP32 numbers, added with Knuth's error-free
// TwoSum, carries ~2^-44 relative accuracy on the FP32 pipe; the FP64 pipe of this
// part (1/64 of FP32, 64-cycle dependent latency) is kept off the reduction chain.
struct f2sum {
    float hi, lo;
};
__device__ __forceinline__ f2sum two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ f2sum f2_add(f2sum a, float b) {
    const f2sum t = two_sum(a.hi, b);
    const float lo = t.lo + a.lo;
    const float hi = t.hi + lo;
    return {hi, lo - (hi - t.hi)};
}
__device__ __forceinline__ f2sum f2_add(f2sum a, f2sum b) {
    const f2sum t = two_sum(a.hi, b.hi);
    const float lo = t.lo + (a.lo + b.lo);
    const float hi = t.hi + lo;
    return {hi, lo - (hi - t.hi)};
}
// Sum of K (a power of two) double-float partials p[0], p[s], ..., p[(K - 1) s] as a balanced
// tree: log2(K) dependent additions instead of K - 1, in an order fixed by K.
template <int K> __device__ __forceinline__ f2sum f2_tree(const f2sum* p, int s) {
    if constexpr (K == 1)
        return p[0];
    else
        return f2_add(f2_tree<K / 2>(p, s), f2_tree<K / 2>(p + (K / 2) * s, s));
}
// k in {1, 2, 4, 8, 16} as the balanced tree; any other k (1..16) as a left fold, also in a fixed order.
__device__ __forceinline__ f2sum f2_tree_sum(const f2sum* p, int k, int s) {
    switch (k) {
        case 16: return f2_tree<16>(p, s);
        case 8: return f2_tree<8>(p, s);
        case 4: return f2_tree<4>(p, s);
        case 2: return f2_tree<2>(p, s);
        case 1: return p[0];
        default: {
            f2sum a = p[0];
            for (int r = 1; r < k; ++r) a = f2_add(a, p[r * s]);
            return a;
        }
    }
}
// Pin a loaded value in a register at this point: the load must complete here, so the
// compiler cannot sink it to its use after the pair loop (where its latency would show).
__device__ __forceinline__ void pin(double v) { asm volatile("" ::"d"(v)); }
__device__ __forceinline__ void pin(float v) { asm volatile("" ::"f"(v)); }
__device__ __forceinline__ void pin(long long v) { asm volatile("" ::"l"(v)); }

// Asynchronous global -> shared copies (cp.async) for the force epilogue's inputs.
struct __align__(16) EpiSlot {
    float4 nz;       // Langevin noise of the next step (times sqrt(T))
    double v[3], x[3], hs, m, o[3];
    float sig0;
    float pad[3];
};
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------------------- pass helpers
// Programmatic dependent launch: let the next kernel in the stream be scheduled
// early, and wait for the previous one before touching what it wrote.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Thread-block-cluster barrier in two halves (every thread of every CTA takes part).
__device__ __forceinline__ void cluster_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_arrive_release() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// Pushing partial sums to the cluster's rank-0 CTA without a second cluster barrier. Rank 0 sets up an
// mbarrier that completes when the expected number of bytes has arrived (and its own single arrival,
// made at set-up); the other CTAs write their partials into rank 0's shared memory with st.async, whose
// completion counts those bytes on that mbarrier, and exit. Rank 0 waits on the mbarrier with a bounded
// number of polls.
__device__ __forceinline__ void mbar_setup(uint64_t* bar, uint32_t tx_bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(tx_bytes) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Shared-memory address of p in the cluster's rank-0 CTA (a shared::cluster address).
__device__ __forceinline__ unsigned rank0_addr(const void* p) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return r;
}
__device__ __forceinline__ void st_async(unsigned raddr, float v, unsigned rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(raddr), "f"(v),
                 "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async(unsigned raddr, double v, unsigned rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(raddr), "d"(v),
                 "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async(unsigned raddr, f2sum v, unsigned rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(v.hi), "f"(v.lo), "r"(rbar)
                 : "memory");
}
// Wait for phase 0 of the mbarrier; false after kMbarPolls polls (each try_wait may also suspend the
// thread for a while), which no correct run comes near: the pushes of a pass land within microseconds.
constexpr int kMbarPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait0(uint64_t* bar) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    for (int k = 0; k < kMbarPolls; ++k) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a)
            : "memory");
        if (done) return true;
    }
    return false;
}
// Status bit set when a bounded wait gave up (reported as MD_ERR_TIMEOUT).
constexpr int kStatusTimeout = 16;

// CTA barrier 1 over the first n threads (n a multiple of 32); barrier 0 is __syncthreads.
__device__ __forceinline__ void bar_sync_first(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

// The work item of this CTA: a table entry, or (one cluster per context) computed in place.
template <int BI> __device__ __forceinline__ Item load_item(const Dev& d, const Item* items, int C) {
    const int k = blockIdx.x / C;
    if (d.single_n > 0) {
        Item it;
        it.i0 = k * BI;
        it.ni = min(BI, d.single_n - it.i0);
        it.j0 = 0;
        it.nj = d.single_n;
        it.cl = 0;
        it.pad = 0;
        return it;
    }
    return items[k];
}

// Every kernel is launched with programmatic stream serialization (it waits on its
// predecessor with griddepcontrol.wait) and, when C > 0, as clusters of C CTAs.
template <class K, class... Args>
inline cudaError_t launch_ex(K kernel, int grid, int threads, size_t smem, int C, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
    if (C > 0) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = C;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <class K, class... Args>
inline cudaError_t launch_cluster(K kernel, int grid, int threads, size_t smem, int C, cudaStream_t s, Args... args) {
    return launch_ex(kernel, grid, threads, smem, C, s, args...);
}

}  // namespace scmd
