// scmd_internal.cuh -- internal types shared by the kernels and the host API of libscmd.
//
// Data layout in HBM (per context; Ntot real atoms, Npad padded):
//   * every cluster's atoms occupy a contiguous padded segment whose length is
//     a multiple of kPad (64) so that 32- and 64-atom i-blocks and 32-atom
//     j-tiles never straddle two clusters;
//   * FP64 state (positions x, velocities v) in structure-of-arrays form
//     x[3][Npad], v[3][Npad]; masses m[Npad];
//   * forces F[3][Npad] in the pass precision (float for MIXED, double for FP64);
//   * "mirror": the positions the density pass reads. MIXED: float4(x - o, 0)
//     with o a per-cluster origin fixed when the context is created (the centre
//     of mass of the initial positions; md_recenter moves it), so forces are a
//     pure function of x for the life of the context (bitwise checkpoint/resume).
//     FP64: the absolute positions as double4;
//   * "posg": what the force pass reads, (x, y, z, B6 * rho^-1/2) per atom,
//     written by the density pass;
//   * rho[Npad] (FP64) and per-32-atom-group observable partials.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace scmd {

constexpr int kPad = 64;        // per-cluster padding granularity (atoms)
constexpr int kGroup = 32;      // atoms per observable partial record (one warp)
constexpr int kObsFields = 16;  // doubles per observable partial record
constexpr int kMaxWarps = 16;
constexpr int kMaxCluster = 8;
constexpr int kCellCap = 256;   // atoms a cell of the cell-list path can hold
constexpr int kVMax = 512;      // entries a neighbour list can hold
constexpr int kVLog = 3;        // a list is split into kVLanes sub-lists, one per thread of its atom
constexpr int kVLanes = 1 << kVLog;
constexpr int kQMax = 2048;     // atoms a quad's neighbour list can hold (MIXED lists)
constexpr float kQuadFar = 1.0e5f;  // MIXED lists: offset of an empty slot (the padding quad's slots sit at -kQuadFar)

// Fields of an observable partial record (per 32-atom group).
enum ObsField {
    OF_EEMB = 0,   // sum over the group of -eps c sqrt(rho_i)                (eV)
    OF_EPAIR = 1,  // sum over the group of sum_j r_ij^-n   (times 1/2 eps a^n later)
    OF_KE2 = 2,    // sum m v^2                                               (amu A^2/fs^2)
    OF_P = 3,      // sum m v (3)
    OF_MX = 6,     // sum m x (3), absolute frame
    OF_L = 9,      // sum m x cross v (3), absolute frame
    OF_MASS = 12,  // sum m
    OF_BAD = 13,   // number of non-finite values seen
};

// One work item of a pair pass: an i-block of one cluster.
struct Item {
    int32_t i0;   // padded global index of the first i atom
    int32_t ni;   // real atoms in this block (<= 32 * ipt)
    int32_t j0;   // padded global index of the cluster's first atom
    int32_t nj;   // real atoms in the cluster
    int32_t cl;   // cluster index
    int32_t pad;
};

// Cell grid of one cluster (cell-list path): G^3 cubic cells of side h >= rcut covering
// the cube [-E, E)^3 around the cluster's origin; cells off .. off + G^3 - 1 of the context.
// h is a binary32 value and E = G h / 2, so the offset between two cell centres, (k - l) h
// with |k - l| <= 1 per axis, is exact in FP32.
struct CellGrid {
    int32_t G, off;
    double h, E, inv_h;
};

// Derived potential constants.
struct Pot {
    double eps, c, a, rcut, rcut2;
    int n, m;
    double A9;   // eps * n * a^n        (force, repulsive part)
    double B6;   // eps * c * m / 2 * a^m (force, embedding part; multiplies rho^-1/2)
    double am;   // a^m                  (density scale)
    double ecoef;// 1/2 eps a^n          (pair energy scale)
    float A9f, rcut2f;
    float gsf;   // B6 / sqrt(a^m) in FP32: g_i = gsf * (sum_j r_ij^-m)^-1/2 without forming rho
    int special; // 1 when (n, m) = (9, 6): compile-time exponents
    int shift;   // 1: every pair term inside rcut less its value at rcut
    double shm;  // rcut^-m: the density shift per pair (rho = a^m (sum r^-m - shm * pairs))
    double shn;  // rcut^-n: the pair-energy shift per pair
};

// Integrator / thermostat parameters of the current md_step call (device resident).
struct Run {
    double dt, h;            // step, half step (fs)
    double hk;               // h (1 + c1): the BAOAB position update as one multiply-add
    double c1;               // Langevin exp(-gamma dt)
    double noise_k;          // (1 - c1^2) k_B * conv  (sigma_i^2 = noise_k * T / m_i)
    double T0, T1;           // ramp end points
    double dT;               // (T1 - T0) / nsteps
    double dt_over_tau;      // Berendsen
    double kb;               // k_B
    int64_t step0;           // global step at the start of the call
    int64_t nsteps;          // steps of the call
    uint64_t seed;
    int32_t kind;            // md_thermo_kind
    int32_t obs_every;       // 0 = never
    int32_t hist_cap;        // ring capacity (samples)
    int32_t pad;
};

// Everything a kernel needs, passed by value.
struct Dev {
    int32_t B;           // clusters
    int32_t npad;        // padded atoms
    int32_t ngroups;     // npad / 32
    int32_t prec;        // md_precision
    int32_t single_n;    // atoms of the only cluster when B == 1 (work items computed in place), else 0
    const int32_t* poff; // [B+1] padded offsets
    const int32_t* nreal;// [B] real atoms per cluster
    const int32_t* cl_of_group; // [ngroups] cluster of each 32-atom group
    double* x;           // [3][npad]
    double* v;           // [3][npad]
    const double* mass;  // [npad]
    void* f;             // [3][npad] float or double
    void* mirror;        // float4 / double4 [npad]
    void* posg;          // float4 / double4 [npad]
    double* rho;         // [npad]
    double* origin;      // [B][3] MIXED mirror origin; FP64: unused
    const double* hs;    // [npad] half-step kick factor h * conv / m (per md_step call)
    const float* sig0;   // [npad] sqrt((1 - c1^2) k_B conv / m) (Langevin, per md_step call)
    float4* noise;       // [noise_steps][npad] Langevin normals of the running chunk times sqrt(T(step)) (MIXED)
    double* part;        // [ngroups][kObsFields]
    double* ke_grp;      // [ngroups] sum m v^2 (Berendsen)
    double* hist;        // ring [cap][B][kHistFields]
    int64_t* step_base;  // [1] global step of local step 0 of the running chunk
    int32_t* status;     // [1] bit 0: non-finite value; bit 1: a cell overflowed
    Run* run;            // device copy of Run
    Pot pot;
    double conv;         // (eV/amu) in (A/fs)^2
    // cell-list path (path == 1); unused by the all-pairs path
    int32_t path;        // 0: all pairs, 1: cell list
    int32_t n_cells;     // cells of all clusters
    const CellGrid* grid;// [B]
    const int32_t* cell_cl;  // [n_cells] cluster of each cell
    const int32_t* cell_order; // [n_cells] pair-pass launch order: cells nearest their cluster's centre first
    int32_t* cell_count; // [n_cells] atoms binned into each cell (may exceed kCellCap: overflow)
    int32_t* cell_atoms; // [n_cells][kCellCap] padded atom indices, ascending within a cell
    int32_t* cell_oct;   // [n_cells][9] first place of each octant of the cell in its sorted slots, then the count
    uint8_t* cell_obyte; // [n_cells][kCellCap] octant of each binned atom, in bin (unsorted) order
    void* cpos;          // [n_cells][kCellCap] V4 (x - cell centre, 0) in the pass precision
    void* cposg;         // [n_cells][kCellCap] V4 (x - cell centre, B6 rho^-1/2), density pass (between the
                         // bin and sort kernels: the offsets in bin order)
    double* eatom;       // [npad][2] per-atom -eps c sqrt(rho_i) and sum_j r_ij^-n
    double* obs_x;       // [npad][3] positions at an observation (end of the step)
    double* obs_v;       // [npad][3] velocities at an observation
    // neighbour-list path (path == 2): per-atom lists of the atoms closer than rcut + skin at the
    // last rebuild, rebuilt when some atom has moved more than skin / 2 since
    int32_t nslot;       // list slots (the real atoms, in cell order at the last rebuild)
    float vskin2h;       // (skin / 2)^2
    double vrl2;         // (rcut + skin)^2
    int32_t* vlist;      // FP64: [nslot][kVMax] slots of the neighbours, by (atom mod kVLanes, atom)
    int32_t* vcount;     // FP64: [nslot]
    int32_t* vsub;       // FP64: [nslot][kVLanes] end of each sub-list (the entries j with j mod kVLanes = t)
    int32_t* vrcount;    // FP64: [nslot] entries of the reverse list (lower atoms that list this one)
    uint64_t* vrev;      // FP64: [nslot][kVMax] reverse list: (lower atom's residue and index, its entry's place)
    int32_t* vrsub;      // FP64: [nslot][kVLanes] end of each residue class of the reverse list
    double* hbuf;        // FP64: [nslot][kVMax] density term of each listed pair, for the partner
    double4* fbuf;       // FP64: [nslot][kVMax] force on the listing atom and pair energy term of each pair
    int2* vcl;           // FP64: [nslot][kVMax] entries inside rcut this step, in list order: (partner, place)
    int32_t* vcn;        // FP64: [nslot] their number
    uint8_t* vflag;      // FP64: [nslot][kVMax] 1 where the list entry's pair is inside rcut this step
    double* rho_half;    // FP64: [nslot] the listing atom's own density sum
    double4* fhalf;      // FP64: [nslot] the listing atom's own force and pair-energy sums
    int32_t* vorder;     // [nslot] atom of each slot (MIXED: -1 for the empty slots that pad cells to quads)
    int32_t* vslotof;    // [npad] slot of each atom
    int32_t* vslot;      // FP64: [1] slot counter of a rebuild
    void* vhi;           // [nslot] by slot: FP64 double4 (x, y, z, 0); MIXED float4 (offset from the quad's
                         // reference point, 0)
    void* vposg;         // [nslot] (vhi.xyz, B6 rho^-1/2), written by the density pass; MIXED a 32-byte record:
                         // that float4, then the quad's reference point (float4, written at the rebuild)
    double* vxref;       // [3][nslot] positions at the last rebuild
    uint32_t* vdmax;     // [2] largest squared displacement since the rebuild (float bits), by step parity
    // MIXED neighbour lists are kept per quad (4 consecutive slots of one cell, from a bisection of its
    // atoms; cells padded to whole quads with empty slots, vorder = -1). nslot = 4 * nqmax there.
    int32_t nqmax;       // quads allocated
    int32_t* q_n;        // [1] quads in use since the last rebuild
    int32_t* cell_base;  // [n_cells + 1] first slot of each cell, then the end of the last
    float4* q_ref;       // [nqmax] reference point of each quad relative to the origin (a multiple of 2^-12 A)
    float4* q_box;       // [nqmax][2] bounding box (lo, hi) of its atoms at the rebuild, relative to the origin
    int32_t* q_cell;     // [nqmax] cell of each quad
    int32_t* q_list;     // [nqmax][kQMax] the slots of the atoms, not of the quad, within rcut + skin of one of
                         // its atoms at the rebuild (lanes past a list's end read the padding quad nqmax,
                         // reference point 0, its 4 slots at -kQuadFar)
    int32_t* q_count;    // [nqmax]
    // FP64 all pairs with each pair evaluated once (scmd_half64.cu); h_nunits == 0: ordered pairs
    int32_t h_nunits;    // work units: (i-tile of 32 atoms, j half-tile of 16) with the half-tile at or after the i-tile
    const int4* h_unit;  // [h_nunits] (first i atom, first j atom, 1 if the half-tile is inside the i-tile, cluster)
    const int32_t* h_ubase;  // [B] first unit of each cluster (units ordered by cluster, i-tile, half-tile)
    void* h_pi;          // [h_nunits][32] dbl4 i-side sums of each unit (density: .x; force: F, sum r^-n)
    void* h_pj;          // [h_nunits][16] dbl4 j-side sums of each unit
};

constexpr int kHistFields = 20;  // doubles per history record (see md_obs packing in the API)

// ---------------------------------------------------------------- launchers
struct Shape { int ipt, warps, cluster; };

// Kernels are launched through these wrappers (defined in scmd_kernels.cu).
cudaError_t launch_mirror(const Dev& d, cudaStream_t s);
cudaError_t launch_origin(const Dev& d, cudaStream_t s);
cudaError_t launch_prepare(const Dev& d, cudaStream_t s);
cudaError_t launch_noise(const Dev& d, int M, cudaStream_t s);
cudaError_t launch_density(const Dev& d, const Item* items, int nitems, Shape sh, int obs, cudaStream_t s);
// mode: 0 = forces only (store F), 1 = forces + all observable partials (no integration),
//       2 = MD step: finish the half kick, record observables if due, start the next step unless last.
// flags (mode 2): bit 0 = last step of the chunk, bit 1 = observables are due at the end of this step.
cudaError_t launch_force(const Dev& d, const Item* items, int nitems, Shape sh, int mode, int k_local,
                         int flags, cudaStream_t s);
cudaError_t launch_start(const Dev& d, int k_local, cudaStream_t s);
cudaError_t launch_berendsen(const Dev& d, int k_local, int last, cudaStream_t s);
cudaError_t launch_obs_reduce(const Dev& d, int k_local, int slot_mode, cudaStream_t s);
cudaError_t launch_advance(const Dev& d, int nsteps, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int n, cudaStream_t s);
cudaError_t launch_normals(uint64_t seed, uint32_t cluster, int64_t step, int n, int prec, double* out,
                           cudaStream_t s);
size_t pass_smem_bytes(int prec, Shape sh, int which);  // which: 0 density pass, 1 force pass
// Cell-list path (defined in scmd_cells.cu).
// clear, bin, sort; cond != 0: only when a neighbour-list rebuild is due at local step k_local
// clear (unless clear == false: MIXED lists inside a step, where k_q_order left the counts clear), bin, sort
cudaError_t launch_cell_build(const Dev& d, cudaStream_t s, int cond = 0, int k_local = 0, bool clear = true);
cudaError_t launch_cell_density(const Dev& d, int obs, cudaStream_t s);
cudaError_t launch_cell_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s);
// Observable partials of every 32-atom group from the per-atom data (from_state: read x, v;
// else the snapshot obs_x, obs_v); with_velocity 0 leaves the velocity fields alone.
cudaError_t launch_cell_obs(const Dev& d, int from_state, int with_velocity, cudaStream_t s);
cudaError_t launch_cell_ke(const Dev& d, cudaStream_t s);
// Neighbour-list path (defined in scmd_verlet.cu).
cudaError_t launch_v_pos(const Dev& d, int k_local, cudaStream_t s);
cudaError_t launch_v_rebuild(const Dev& d, int cond, int k_local, cudaStream_t s);  // after the cell build
cudaError_t launch_v_density(const Dev& d, int obs, cudaStream_t s, int k_local = -1);  // k_local: MD step
cudaError_t launch_v_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s);
// MIXED quad lists (defined in scmd_quads.cu); launch_v_* dispatch to them for MIXED.
cudaError_t launch_q_pos(const Dev& d, int k_local, cudaStream_t s);
cudaError_t launch_q_rebuild(const Dev& d, int cond, int k_local, cudaStream_t s);  // after the cell build
cudaError_t launch_q_density(const Dev& d, int obs, int k_local, cudaStream_t s);  // k_local < 0: outside a step
cudaError_t launch_q_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s);
// Structural observables (defined in scmd_structure.cu).
constexpr int kNbCap = 32;  // neighbours a CNA list stores (the count is exact beyond)
struct StructBufs {
    double* com;               // [B][3]
    int32_t* core;             // [npad] core atoms of each cluster, from its padded offset on
    int32_t* ncore;            // [B]
    unsigned long long* hist;  // [B][nbins]
    double* ref;               // [3][npad] reference positions of the displacement
    double* ref_com;           // [B][3]
    uint8_t* sel;              // [npad] atoms the displacement averages over
    double* msd;               // [B]
    int32_t* nsel;             // [B]
    int32_t* nb;               // [npad][kNbCap] neighbours, ascending
    int32_t* nnb;              // [npad]
    int8_t* cls;               // [npad] 0 other, 1 fcc, 2 hcp, 3 icosahedral
    int32_t* counts;           // [B][4] atoms of each class
    int32_t* capped;           // [B] atoms left "other" because a neighbour had more than kNbCap neighbours
};
// Y CTAs per cluster share its pair-distance histogram.
cudaError_t launch_rdf(const Dev& d, const StructBufs& sb, double r_core, double width, int nbins, int Y,
                       cudaStream_t s);
cudaError_t launch_msd_ref(const Dev& d, const StructBufs& sb, double r_core, cudaStream_t s);
cudaError_t launch_msd(const Dev& d, const StructBufs& sb, cudaStream_t s);
cudaError_t launch_cna(const Dev& d, const StructBufs& sb, double r_nb, cudaStream_t s);
// FP64 all pairs, each pair once (defined in scmd_half64.cu): pair kernel + per-atom sum kernel per pass.
cudaError_t launch_h_density(const Dev& d, int obs, cudaStream_t s);
cudaError_t launch_h_force(const Dev& d, int mode, int k_local, int flags, cudaStream_t s);
// State exchange with caller-owned device arrays (defined in scmd_import.cu). off[B+1] are the
// unpadded cluster offsets of the caller's [Ntot][3] / [Ntot] arrays.
int invalid_input_bit();  // status bit launch_check_input sets
cudaError_t launch_check_input(const double* pos, const double* vel, const double* mass, int64_t ntot,
                               int32_t* status, cudaStream_t s);
cudaError_t launch_import(const Dev& d, const int32_t* off, const double* pos, const double* vel,
                          const double* mass, cudaStream_t s);
cudaError_t launch_export(const Dev& d, const int32_t* off, double* pos, double* vel, cudaStream_t s);
// forces (caller layout, doubles) and per-cluster potential energies from history slot hist_slot
cudaError_t launch_export_forces(const Dev& d, const int32_t* off, double* forces, double* epot, int hist_slot,
                                 cudaStream_t s);
// The calling thread's error message returned by md_last_error(NULL) (defined in scmd_api.cu).
void set_thread_error(const char* msg);
cudaError_t configure_kernels();

}  // namespace scmd
