// scmd_import.cu -- state exchange with caller-owned device arrays (md_create_device,
// md_set_state_device, md_get_state_device, md_energy_forces_device).
//
// The caller's arrays are row-major [Ntot][3] doubles (positions, velocities) and [Ntot]
// doubles (masses) in device memory, clusters back to back. The context keeps the padded
// structure-of-arrays layout x[3][Npad] (see scmd_internal.cuh); these kernels convert
// between the two on the context's stream, so a PyTorch caller never stages the state
// through host memory.
#include <algorithm>

#include "scmd_internal.cuh"

namespace scmd {
namespace {

// Bit of the context status word set by k_check_input when an input value is invalid.
constexpr int kInvalidInputBit = 8;

// Every position (and velocity, when given) finite; every mass (when given) finite and > 0.
__global__ void k_check_input(const double* __restrict__ pos, const double* __restrict__ vel,
                              const double* __restrict__ mass, int64_t ntot, int32_t* status) {
    bool bad = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ntot; k += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            bad |= !isfinite(pos[3 * k + c]);
            if (vel) bad |= !isfinite(vel[3 * k + c]);
        }
        if (mass) bad |= !(isfinite(mass[k]) && mass[k] > 0.0);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kInvalidInputBit);
}

// Caller layout -> context layout, one thread per padded atom. Padding atoms get x = v = 0 and
// mass 1 (as md_create sets them). vel == NULL: zero velocities; mass == NULL: masses untouched.
__global__ void k_import(const Dev d, const int32_t* __restrict__ off, const double* __restrict__ pos,
                         const double* __restrict__ vel, const double* __restrict__ mass) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.npad) return;
    const int cl = d.cl_of_group[p >> 5];
    const int a = p - d.poff[cl];
    const bool real = a < d.nreal[cl];
    const int64_t s = (int64_t)off[cl] + a;
    const int np = d.npad;
    for (int c = 0; c < 3; ++c) {
        d.x[c * np + p] = real ? pos[3 * s + c] : 0.0;
        d.v[c * np + p] = (real && vel) ? vel[3 * s + c] : 0.0;
    }
    if (mass) const_cast<double*>(d.mass)[p] = real ? mass[s] : 1.0;
}

// Context layout -> caller layout (positions and/or velocities).
__global__ void k_export(const Dev d, const int32_t* __restrict__ off, double* __restrict__ pos,
                         double* __restrict__ vel) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.npad) return;
    const int cl = d.cl_of_group[p >> 5];
    const int a = p - d.poff[cl];
    if (a >= d.nreal[cl]) return;
    const int64_t s = (int64_t)off[cl] + a;
    const int np = d.npad;
    for (int c = 0; c < 3; ++c) {
        if (pos) pos[3 * s + c] = d.x[c * np + p];
        if (vel) vel[3 * s + c] = d.v[c * np + p];
    }
}

// Forces (context layout, FP32 in MIXED or FP64) -> caller layout [Ntot][3] doubles, and each cluster's
// potential energy from the observables record of the last fresh evaluation.
template <int PREC>
__global__ void k_export_forces(const Dev d, const int32_t* __restrict__ off, double* __restrict__ forces,
                                double* __restrict__ epot, int hist_slot) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (epot && p < d.B) epot[p] = d.hist[((size_t)hist_slot * d.B + p) * kHistFields];
    if (!forces || p >= d.npad) return;
    const int cl = d.cl_of_group[p >> 5];
    const int a = p - d.poff[cl];
    if (a >= d.nreal[cl]) return;
    const int64_t s = (int64_t)off[cl] + a;
    const int np = d.npad;
    for (int c = 0; c < 3; ++c)
        forces[3 * s + c] = PREC == 1 ? (double)reinterpret_cast<const float*>(d.f)[c * np + p]
                                      : reinterpret_cast<const double*>(d.f)[c * np + p];
}

}  // namespace

int invalid_input_bit() { return kInvalidInputBit; }

cudaError_t launch_export_forces(const Dev& d, const int32_t* off, double* forces, double* epot, int hist_slot,
                                 cudaStream_t s) {
    const int n = d.npad > d.B ? d.npad : d.B;
    if (d.prec == 1)
        k_export_forces<1><<<(n + 255) / 256, 256, 0, s>>>(d, off, forces, epot, hist_slot);
    else
        k_export_forces<0><<<(n + 255) / 256, 256, 0, s>>>(d, off, forces, epot, hist_slot);
    return cudaGetLastError();
}

cudaError_t launch_check_input(const double* pos, const double* vel, const double* mass, int64_t ntot,
                               int32_t* status, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((ntot + 255) / 256, 152 * 8);
    k_check_input<<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(pos, vel, mass, ntot, status);
    return cudaGetLastError();
}

cudaError_t launch_import(const Dev& d, const int32_t* off, const double* pos, const double* vel,
                          const double* mass, cudaStream_t s) {
    k_import<<<(d.npad + 255) / 256, 256, 0, s>>>(d, off, pos, vel, mass);
    return cudaGetLastError();
}

cudaError_t launch_export(const Dev& d, const int32_t* off, double* pos, double* vel, cudaStream_t s) {
    k_export<<<(d.npad + 255) / 256, 256, 0, s>>>(d, off, pos, vel);
    return cudaGetLastError();
}

}  // namespace scmd
