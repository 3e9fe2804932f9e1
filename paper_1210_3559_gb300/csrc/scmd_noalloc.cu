// scmd_noalloc.cu -- md_energy_forces_noalloc: energy and forces of one cluster without
// allocating any device memory.
//
// Some callers cannot allocate: a host framework whose own allocator owns all device
// memory and forbids others from calling cudaMalloc, or a time-critical loop that must
// never enter the CUDA allocator. For them this entry point takes caller-owned device
// buffers for its input (positions) and outputs (forces, energy) and keeps its working
// data (the cluster origin, FP32 pair coordinates, rho^-1/2 and per-atom energy terms) in
// one file-scope __device__ array of fixed size (kNoAllocMaxAtoms atoms, about 0.77 MB)
// that every GPU loading this library holds until the process exits.
//
// The arithmetic is that of md_energy_forces in MIXED precision (FP32 pair terms on
// FP32 offsets from the centre of mass, FP64 accumulation of rho and of the energy), with
// a plain tiled layout: one i-atom per thread, j-tiles staged in shared memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/scmd.h"
#include "scmd_internal.cuh"

namespace {

constexpr int kNoAllocMaxAtoms = 16384;
constexpr int kThreads = 128;

struct NoAllocScratch {
    double origin[4];                    // centre of mass of the positions
    float4 mirror[kNoAllocMaxAtoms];     // (x - o, y - o, z - o, 0) in FP32
    float4 posg[kNoAllocMaxAtoms];       // (x, y, z, B * rho^-1/2)
    double e_emb[kNoAllocMaxAtoms];      // -eps c sqrt(rho_i)
    double e_pair[kNoAllocMaxAtoms];     // sum_j r_ij^-n
};

// Shared by every call on a device; each call overwrites what it reads before reading it.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the scratch array per device ordinal, with the id of the CUDA context it was
// looked up in: a device reset makes a new primary context, reloads the module, and may move the
// array, so a changed context id means the address is looked up again.
struct ScratchAddr {
    NoAllocScratch* ptr;
    unsigned long long ctx_id;
    bool have_id;
};
std::mutex g_noalloc_mutex;
ScratchAddr g_noalloc_addr[256] = {};

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current CUDA context (through the driver entry points the runtime
// exposes, so the library needs no link to the driver library); false when unavailable.
bool current_ctx_id(unsigned long long* id) {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PfnCtxGetId>(f);
    }
    CUcontext cur = nullptr;
    if (!get_current || !get_id || get_current(&cur) != CUDA_SUCCESS || !cur) return false;
    return get_id(cur, id) == CUDA_SUCCESS;
}

struct Consts {
    double eps, c, a, am, B, A, ecoef, rcut2;
    int n, m, cut;
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float powr(float inv, float ir, int k) {
    float p = 1.0f;
    for (int e = 0; e < (k >> 1); ++e) p *= inv;
    return (k & 1) ? p * ir : p;
}

// Centre of mass (equal masses: the positions' mean) of the cluster, one CTA, fixed order.
__global__ void k_na_origin(NoAllocScratch* S, const double* pos, int n) {
    __shared__ double sh[kThreads];
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int c = 0; c < 3; ++c) s[c] += pos[3 * i + c];
    for (int c = 0; c < 3; ++c) {
        const double t = block_sum(s[c], sh);
        if (threadIdx.x == 0) S->origin[c] = t / n;
    }
}

__global__ void k_na_mirror(NoAllocScratch* S, const double* pos, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    S->mirror[i] = make_float4((float)(pos[3 * i] - S->origin[0]), (float)(pos[3 * i + 1] - S->origin[1]),
                               (float)(pos[3 * i + 2] - S->origin[2]), 0.f);
}

// rho_i = a^m sum_{j != i} r_ij^-m (Eq. 2); FP32 terms summed per 128-atom tile, tiles in FP64.
__global__ void k_na_density(NoAllocScratch* S, int n, Consts K) {
    __shared__ float4 tile[kThreads];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float4 pi = i < n ? S->mirror[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float rc2 = (float)K.rcut2;
    double rho = 0.0;
    for (int j0 = 0; j0 < n; j0 += kThreads) {
        __syncthreads();
        if (j0 + (int)threadIdx.x < n) tile[threadIdx.x] = S->mirror[j0 + threadIdx.x];
        __syncthreads();
        const int nv = min(kThreads, n - j0);
        float acc = 0.f;
        for (int k = 0; k < nv; ++k) {
            const float dx = pi.x - tile[k].x, dy = pi.y - tile[k].y, dz = pi.z - tile[k].z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (j0 + k == i || (K.cut && !(r2 < rc2))) continue;
            const float ir = rsqrtf(r2);
            acc += powr(ir * ir, ir, K.m);
        }
        rho += (double)acc;
    }
    if (i >= n) return;
    rho *= K.am;
    S->posg[i] = make_float4(pi.x, pi.y, pi.z, rho > 0.0 ? (float)(K.B / sqrt(rho)) : 0.f);
    S->e_emb[i] = -K.eps * K.c * sqrt(rho);
}

// F_i = sum_{j != i} r^-2 [A r^-n - B (g_i + g_j) r^-m] (r_i - r_j) (-dU/dr_i of Eq. 1).
__global__ void k_na_force(NoAllocScratch* S, int n, Consts K, double* forces) {
    __shared__ float4 tile[kThreads];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float4 pi = i < n ? S->posg[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float A = (float)K.A, rc2 = (float)K.rcut2;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    double ep = 0.0;
    for (int j0 = 0; j0 < n; j0 += kThreads) {
        __syncthreads();
        if (j0 + (int)threadIdx.x < n) tile[threadIdx.x] = S->posg[j0 + threadIdx.x];
        __syncthreads();
        const int nv = min(kThreads, n - j0);
        float tx = 0.f, ty = 0.f, tz = 0.f, te = 0.f;
        for (int k = 0; k < nv; ++k) {
            const float4 p = tile[k];
            const float dx = pi.x - p.x, dy = pi.y - p.y, dz = pi.z - p.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (j0 + k == i || (K.cut && !(r2 < rc2))) continue;
            const float ir = rsqrtf(r2), inv = ir * ir;
            const float rn = powr(inv, ir, K.n), rm = powr(inv, ir, K.m);
            const float coef = inv * (A * rn - (pi.w + p.w) * rm);
            tx = fmaf(coef, dx, tx);
            ty = fmaf(coef, dy, ty);
            tz = fmaf(coef, dz, tz);
            te += rn;
        }
        fx += tx;
        fy += ty;
        fz += tz;
        ep += (double)te;
    }
    if (i >= n) return;
    forces[3 * i] = (double)fx;
    forces[3 * i + 1] = (double)fy;
    forces[3 * i + 2] = (double)fz;
    S->e_pair[i] = ep;
}

// U = sum_i [ 1/2 eps a^n e_pair_i + e_emb_i ] (Eq. 1), one CTA, fixed order.
__global__ void k_na_energy(NoAllocScratch* S, int n, Consts K, double* epot) {
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += K.ecoef * S->e_pair[i] + S->e_emb[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) epot[0] = s;
}

// Failures are reported through md_last_error(NULL), like md_create's.
md_status na_fail(md_status st, const char* msg) {
    scmd::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" {

md_status md_energy_forces_noalloc(const double* pos_dev, int32_t n_atoms, const md_sc_params* params,
                                   double* forces_dev, double* epot_dev, uint64_t stream) {
    scmd::set_thread_error("");
    if (!pos_dev || !params || !forces_dev || !epot_dev) return na_fail(MD_ERR_INVALID, "NULL argument");
    if (n_atoms < 1 || n_atoms > kNoAllocMaxAtoms) {
        char buf[160];
        snprintf(buf, sizeof buf, "md_energy_forces_noalloc: n_atoms = %d is outside 1..%d (the fixed scratch size)",
                 n_atoms, kNoAllocMaxAtoms);
        return na_fail(MD_ERR_INVALID, buf);
    }
    if (!(std::isfinite(params->eps_eV) && std::isfinite(params->c) && std::isfinite(params->a_A) &&
          params->a_A > 0 && std::isfinite(params->rcut_A) && params->rcut_A >= 0 && params->n >= 1 &&
          params->n <= 32 && params->m >= 1 && params->m <= 32 && params->reserved == 0))
        return na_fail(MD_ERR_INVALID, "invalid Sutton-Chen parameters");
    if (params->cutoff_shift != 0) return na_fail(MD_ERR_INVALID, "this entry point sums plain (unshifted) terms");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) return na_fail(MD_ERR_CUDA, "no usable CUDA device");
    NoAllocScratch* S = nullptr;
    {
        // first call on this device (or in a new context of it): look up the device address of the
        // scratch array, with this device current
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        ScratchAddr& A = g_noalloc_addr[dev];
        unsigned long long id = 0;
        const bool have_id = current_ctx_id(&id);
        if (!A.ptr || !have_id || !A.have_id || A.ctx_id != id) {
            NoAllocScratch* p = nullptr;
            e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
            if (e != cudaSuccess) {
                A = ScratchAddr{};
                return na_fail(MD_ERR_CUDA, cudaGetErrorString(e));
            }
            A.ptr = p;
            A.have_id = current_ctx_id(&A.ctx_id);  // the lookup has made the context current
        }
        S = A.ptr;
    }
    Consts K;
    K.eps = params->eps_eV;
    K.c = params->c;
    K.a = params->a_A;
    K.n = params->n;
    K.m = params->m;
    K.am = std::pow(K.a, K.m);
    K.A = K.eps * K.n * std::pow(K.a, K.n);
    K.B = K.eps * K.c * K.m * 0.5 * K.am;
    K.ecoef = 0.5 * K.eps * std::pow(K.a, K.n);
    K.cut = params->rcut_A > 0 ? 1 : 0;
    K.rcut2 = params->rcut_A * params->rcut_A;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = (n_atoms + kThreads - 1) / kThreads;
    k_na_origin<<<1, kThreads, 0, s>>>(S, pos_dev, n_atoms);
    k_na_mirror<<<blocks, kThreads, 0, s>>>(S, pos_dev, n_atoms);
    k_na_density<<<blocks, kThreads, 0, s>>>(S, n_atoms, K);
    k_na_force<<<blocks, kThreads, 0, s>>>(S, n_atoms, K, forces_dev);
    k_na_energy<<<1, kThreads, 0, s>>>(S, n_atoms, K, epot_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(MD_ERR_CUDA, cudaGetErrorString(e));
    return MD_OK;
}

}  // extern "C"
