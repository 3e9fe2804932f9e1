// scmd_api.cu -- host side of the libscmd C ABI (declared in include/scmd.h).
//
// A context owns the device-resident state of a batch of clusters and issues,
// per MD step, the density pass and the force pass (whose epilogue integrates),
// preceded on the cell-list path by the cell build (clear, bin, sort), plus a
// Berendsen kernel when that thermostat is selected and an observables
// reduction when a sample is due. md_step replays CUDA graphs that each hold
// one chunk of steps (step start, the kernels of every step, step counter
// advance); graphs are cached by chunk length, the observation phase of the
// chunk's first step, the thermostat kind and the launch shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/scmd.h"
#include "scmd_device.cuh"

using namespace scmd;

namespace {

// (eV/amu) in (A/fs)^2 = e / u * 1e-10 (e exact SI 2019, u CODATA 2018); k_B in eV/K (exact).
constexpr double kConv = 1.602176634e-19 / 1.66053906660e-27 * 1.0e-10;
constexpr double kKB = 8.617333262e-5;

thread_local std::string g_create_error;

// MD_PATH_AUTO with a cutoff takes the cell list once the largest cluster has this many atoms:
// below it the 27 cells of side >= rcut around an atom hold most of the cluster anyway.
constexpr int kAutoCellsMinAtoms = 8192;
// Neighbour-list path: the lists hold the atoms within rcut + kSkin; they are rebuilt when some atom
// has moved more than kSkin / 2 since the last rebuild.
constexpr double kSkin = 1.0;
constexpr double kSkinMargin = 1e-3;  // the rebuild triggers at kSkin / 2 - kSkinMargin (covers rounding)
constexpr double kPi = 3.14159265358979323846;
// MD_PATH_AUTO in FP64 evaluates each pair once when the batch has at least this many work units
// (32 x 16 atoms each): two per FP64 sub-partition of the 152 SMs, i.e. about one 1100-atom
// cluster. Below it the ordered-pair kernels, which spread a small cluster's pairs over more warps,
// finish sooner...
constexpr int kHalfMinUnits = 2 * 4 * 152;
// ... and when its clusters are large: a unit covers 32 x 16 atoms, so for small clusters the ragged
// tiles, and the diagonal units that visit their pairs twice, take much of the work (64 Ni147 clusters:
// the ordered-pair kernels measured 1.65x faster). Pair-weighted mean cluster size, atoms.
constexpr double kHalfMinMeanSize = 512.0;

struct GraphKey {
    int M, phase, kind, obs_every;
    int dens[3], force[3];
    bool operator<(const GraphKey& o) const {
        return std::tie(M, phase, kind, obs_every, dens[0], dens[1], dens[2], force[0], force[1], force[2]) <
               std::tie(o.M, o.phase, o.kind, o.obs_every, o.dens[0], o.dens[1], o.dens[2], o.force[0], o.force[1],
                        o.force[2]);
    }
};

}  // namespace

void scmd::set_thread_error(const char* msg) { g_create_error = msg ? msg : ""; }

struct md_ctx {
    md_config cfg{};
    Pot pot{};
    int B = 0;
    int64_t ntot = 0;
    int npad = 0, ngroups = 0;
    std::vector<int32_t> sizes, off, poff, cl_of_group;
    std::vector<Item> items_h[3];  // ipt 1, 2 and 4 (4: the density pass only)
    Item* items_d[3] = {nullptr, nullptr, nullptr};
    Shape shape[2] = {{1, 4, 1}, {1, 4, 1}};  // density, force
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device buffers
    int32_t *d_poff = nullptr, *d_nreal = nullptr, *d_clg = nullptr, *d_status = nullptr;
    int32_t* d_off = nullptr;  // [B+1] unpadded cluster offsets (caller layout of the state arrays)
    // FP64 all pairs with each pair once (scmd_half64.cu)
    bool half = false;
    int32_t h_nunits = 0;
    int4* d_h_unit = nullptr;
    int32_t* d_h_ubase = nullptr;
    void *d_h_pi = nullptr, *d_h_pj = nullptr;
    double *d_x = nullptr, *d_v = nullptr, *d_mass = nullptr, *d_rho = nullptr, *d_origin = nullptr;
    double *d_part = nullptr, *d_ke = nullptr, *d_hist = nullptr, *d_hs = nullptr;
    float* d_sig0 = nullptr;
    float4* d_noise = nullptr;
    int noise_steps = 0;  // capacity of d_noise in steps (MIXED); chunks never exceed it
    void *d_f = nullptr, *d_mirror = nullptr, *d_posg = nullptr;
    int64_t* d_step = nullptr;
    Run* d_run = nullptr;
    // cell-list path
    int path = 0;  // 0: all pairs, 1: cells
    int n_cells = 0;
    std::vector<CellGrid> grids;
    CellGrid* d_grid = nullptr;
    int32_t *d_cell_cl = nullptr, *d_cell_count = nullptr, *d_cell_atoms = nullptr, *d_cell_order = nullptr;
    int32_t* d_cell_oct = nullptr;
    // structural observables (allocated at first use)
    StructBufs sb{};
    int sb_nbins = 0;
    bool msd_ref = false;
    // neighbour-list path
    int32_t *d_vlist = nullptr, *d_vcount = nullptr, *d_vsub = nullptr, *d_vorder = nullptr, *d_vslotof = nullptr;
    int32_t *d_vslot = nullptr, *d_vrcount = nullptr, *d_vrsub = nullptr, *d_vcn = nullptr;
    int2* d_vcl = nullptr;
    uint8_t* d_vflag = nullptr;
    uint64_t* d_vrev = nullptr;
    double *d_hbuf = nullptr, *d_rho_half = nullptr;
    double4 *d_fbuf = nullptr, *d_fhalf = nullptr;
    void *d_vhi = nullptr, *d_vposg = nullptr;
    int32_t *d_q_n = nullptr, *d_cell_base = nullptr, *d_q_cell = nullptr, *d_q_list = nullptr, *d_q_count = nullptr;
    float4 *d_q_ref = nullptr, *d_q_box = nullptr;
    int nqmax = 0;
    int32_t nslot = 0;  // list slots: the atoms (FP64), or 4 * nqmax (MIXED quads)
    double* d_vxref = nullptr;
    uint32_t* d_vdmax = nullptr;
    uint8_t* d_cell_obyte = nullptr;
    void *d_cpos = nullptr, *d_cposg = nullptr;
    double *d_eatom = nullptr, *d_obs_x = nullptr, *d_obs_v = nullptr;
    // pinned staging
    double* h_stage = nullptr;
    size_t h_stage_n = 0;
    Run* h_run = nullptr;
    int64_t* h_step = nullptr;
    // state
    int64_t step = 0;
    double time_fs = 0.0;
    int hist_cap = 4096;
    std::deque<std::pair<int64_t, double>> samples;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::string err;
    Dev dev{};
};

namespace {

md_status fail(md_ctx* c, md_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define CK(ctx, call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            md_status st_ = (e_ == cudaErrorMemoryAllocation) ? MD_ERR_OOM : MD_ERR_CUDA;         \
            return fail(ctx, st_, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                \
        }                                                                                         \
    } while (0)

// Device memory of a context is allocated and freed in stream order on the context's stream
// (the caller's stream when md_config.stream is set).
template <class T> cudaError_t dmalloc(md_ctx* c, T** p, size_t bytes) {
    return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, c->stream);
}
void dfree(md_ctx* c, void* p) {
    if (!p) return;
    if (c->stream)
        cudaFreeAsync(p, c->stream);
    else
        cudaFree(p);
}

bool finite_all(const double* p, size_t n) {
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(p[k])) return false;
    return true;
}

int elem_size(const md_ctx* c) { return c->cfg.precision == MD_PREC_MIXED ? 4 : 8; }
int vec4_size(const md_ctx* c) { return c->cfg.precision == MD_PREC_MIXED ? 16 : 32; }

void fill_dev(md_ctx* c) {
    Dev& d = c->dev;
    d.B = c->B;
    d.npad = c->npad;
    d.ngroups = c->ngroups;
    d.prec = c->cfg.precision;
    d.single_n = c->B == 1 ? c->sizes[0] : 0;
    d.poff = c->d_poff;
    d.nreal = c->d_nreal;
    d.cl_of_group = c->d_clg;
    d.x = c->d_x;
    d.v = c->d_v;
    d.mass = c->d_mass;
    d.f = c->d_f;
    d.mirror = c->d_mirror;
    d.posg = c->d_posg;
    d.rho = c->d_rho;
    d.origin = c->d_origin;
    d.hs = c->d_hs;
    d.sig0 = c->d_sig0;
    d.noise = c->d_noise;
    d.part = c->d_part;
    d.ke_grp = c->d_ke;
    d.hist = c->d_hist;
    d.step_base = c->d_step;
    d.status = c->d_status;
    d.run = c->d_run;
    d.pot = c->pot;
    d.conv = kConv;
    d.path = c->path;
    d.n_cells = c->n_cells;
    d.grid = c->d_grid;
    d.cell_cl = c->d_cell_cl;
    d.cell_order = c->d_cell_order;
    d.cell_count = c->d_cell_count;
    d.cell_atoms = c->d_cell_atoms;
    d.cell_oct = c->d_cell_oct;
    d.cell_obyte = c->d_cell_obyte;
    d.nslot = c->nslot;
    d.vskin2h = (float)((0.5 * kSkin - kSkinMargin) * (0.5 * kSkin - kSkinMargin));
    d.vrl2 = (c->pot.rcut + kSkin) * (c->pot.rcut + kSkin);
    d.vlist = c->d_vlist;
    d.vcount = c->d_vcount;
    d.vsub = c->d_vsub;
    d.vrcount = c->d_vrcount;
    d.vrev = c->d_vrev;
    d.vrsub = c->d_vrsub;
    d.vcl = c->d_vcl;
    d.vcn = c->d_vcn;
    d.vflag = c->d_vflag;
    d.hbuf = c->d_hbuf;
    d.fbuf = c->d_fbuf;
    d.rho_half = c->d_rho_half;
    d.fhalf = c->d_fhalf;
    d.vorder = c->d_vorder;
    d.vslotof = c->d_vslotof;
    d.vslot = c->d_vslot;
    d.vhi = c->d_vhi;
    d.nqmax = c->nqmax;
    d.q_n = c->d_q_n;
    d.cell_base = c->d_cell_base;
    d.q_ref = c->d_q_ref;
    d.q_box = c->d_q_box;
    d.q_cell = c->d_q_cell;
    d.q_list = c->d_q_list;
    d.q_count = c->d_q_count;
    d.vposg = c->d_vposg;
    d.vxref = c->d_vxref;
    d.vdmax = c->d_vdmax;
    d.cpos = c->d_cpos;
    d.cposg = c->d_cposg;
    d.eatom = c->d_eatom;
    d.obs_x = c->d_obs_x;
    d.obs_v = c->d_obs_v;
    d.h_nunits = c->half ? c->h_nunits : 0;
    d.h_unit = c->d_h_unit;
    d.h_ubase = c->d_h_ubase;
    d.h_pi = c->d_h_pi;
    d.h_pj = c->d_h_pj;
}

// Cell grid of every cluster (cell-list and neighbour-list paths; "rcut" below is the reach:
// rcut, or rcut + skin for the neighbour lists). The cube [-E, E)^3 around the origin covers the
// cluster with a margin: E = max(1.3 R_fcc, 1.1 R_now) + rcut, R_fcc the radius of N atoms at
// the fcc density 4 / a^3 and R_now the largest distance of an atom from the centre of mass
// (clamped to 3 R_fcc so that a few far atoms cannot blow up the grid; those sit in border
// cells). G = floor(2E / rcut) cells per axis (at most 128), side h = 2E / G >= rcut, rounded
// up to a binary32 value (E is then G h / 2) so that offsets between cell centres are exact in FP32.
// Returns false when a cell at the fcc density would not fit kCellCap atoms.
bool make_grids(md_ctx* c, const double* pos, const double* mass, double reach) {
    const double rc = reach, a = c->pot.a;
    c->grids.resize(c->B);
    int off = 0;
    for (int b = 0; b < c->B; ++b) {
        const int n = c->sizes[b];
        const double* x = pos + 3 * (size_t)c->off[b];
        const double* m = mass + c->off[b];
        double com[3] = {0, 0, 0}, M = 0;
        for (int k = 0; k < n; ++k) {
            for (int q = 0; q < 3; ++q) com[q] += m[k] * x[3 * k + q];
            M += m[k];
        }
        for (int q = 0; q < 3; ++q) com[q] /= M;
        double r2max = 0;
        for (int k = 0; k < n; ++k) {
            double r2 = 0;
            for (int q = 0; q < 3; ++q) r2 += (x[3 * k + q] - com[q]) * (x[3 * k + q] - com[q]);
            r2max = std::max(r2max, r2);
        }
        const double r_fcc = a * std::cbrt(3.0 * n / (16.0 * kPi));
        const double r_now = std::min(std::sqrt(r2max), 3.0 * r_fcc);
        const double E = std::max(1.3 * r_fcc, 1.1 * r_now) + rc;
        // (1 + 1e-6): h > rcut strictly, so rounding at a cell face cannot matter
        const int G = std::max(1, std::min(128, (int)std::floor(2.0 * E / (rc * (1.0 + 1e-6)))));
        CellGrid g{};
        g.G = G;
        g.off = off;
        float hf = (float)(2.0 * E / G);
        if ((double)hf < 2.0 * E / G) hf = std::nextafter(hf, 1e30f);
        g.h = (double)hf;
        g.E = 0.5 * G * g.h;
        g.inv_h = 1.0 / g.h;
        // a cell at the fcc density (or the whole cluster, if smaller) must fit kCellCap atoms
        if (std::min(1.25 * 4.0 * g.h * g.h * g.h / (a * a * a), (double)n) > kCellCap) return false;
        c->grids[b] = g;
        off += G * G * G;
    }
    c->n_cells = off;
    return true;
}

Shape default_shape(const md_ctx* c, int which) {
    (void)which;
    const int items = (int)c->items_h[0].size();
    const int target = 152 * 16;  // warps in flight
    Shape s{1, 4, 1};
    int need = (target + items * s.warps - 1) / (items * s.warps);
    while (s.cluster < need && s.cluster < 8) s.cluster *= 2;
    return s;
}

// which: 0 density pass (i-atoms per thread 1, 2 or 4), 1 force pass (1 or 2). A CTA needs at least one
// thread per i-atom of its block (the reduction and the epilogue take one atom per thread): ipt <= warps.
bool shape_ok(Shape s, int which) {
    return (s.ipt == 1 || s.ipt == 2 || (which == 0 && s.ipt == 4)) && s.ipt <= s.warps && (s.warps == 2 || s.warps == 4 || s.warps == 8 || s.warps == 16) &&
           s.cluster >= 1 && s.cluster <= 8;
}

const Item* items_for(const md_ctx* c, Shape s, int* n) {
    const int k = s.ipt == 4 ? 2 : (s.ipt == 2 ? 1 : 0);
    *n = (int)c->items_h[k].size();
    return c->items_d[k];
}

// Host AoS [N][3] <-> padded SoA [3][npad] via the pinned staging buffer.
void pack(const md_ctx* c, const double* aos, double* soa) {
    for (int b = 0; b < c->B; ++b)
        for (int a = 0; a < c->sizes[b]; ++a) {
            const int64_t s = (int64_t)c->off[b] + a;
            const int p = c->poff[b] + a;
            for (int k = 0; k < 3; ++k) soa[(size_t)k * c->npad + p] = aos[3 * s + k];
        }
}
void unpack(const md_ctx* c, const double* soa, double* aos) {
    for (int b = 0; b < c->B; ++b)
        for (int a = 0; a < c->sizes[b]; ++a) {
            const int64_t s = (int64_t)c->off[b] + a;
            const int p = c->poff[b] + a;
            for (int k = 0; k < 3; ++k) aos[3 * s + k] = soa[(size_t)k * c->npad + p];
        }
}

md_status upload_state(md_ctx* c, const double* pos, const double* vel) {
    double* st = c->h_stage;
    std::fill(st, st + 3 * (size_t)c->npad, 0.0);
    pack(c, pos, st);
    CK(c, cudaMemcpyAsync(c->d_x, st, sizeof(double) * 3 * c->npad, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::fill(st, st + 3 * (size_t)c->npad, 0.0);
    if (vel) pack(c, vel, st);
    CK(c, cudaMemcpyAsync(c->d_v, st, sizeof(double) * 3 * c->npad, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return MD_OK;
}

md_status set_step_base(md_ctx* c, int64_t s) {
    *c->h_step = s;
    CK(c, cudaMemcpyAsync(c->d_step, c->h_step, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    return MD_OK;
}

// Forces (and optionally observable partials) of the current positions.
md_status evaluate(md_ctx* c, bool observe) {
    const Dev& d = c->dev;
    int n0, n1;
    const Item* i0 = items_for(c, c->shape[0], &n0);
    const Item* i1 = items_for(c, c->shape[1], &n1);
    CK(c, launch_mirror(d, c->stream));
    if (c->path == 2) {  // lists from the current positions (the results do not depend on when)
        CK(c, launch_cell_build(d, c->stream));
        CK(c, launch_v_rebuild(d, 0, 0, c->stream));
        CK(c, cudaMemsetAsync(c->d_vdmax, 0, sizeof(uint32_t) * 2, c->stream));
        CK(c, launch_v_density(d, observe ? 1 : 0, c->stream));
        CK(c, launch_v_force(d, observe ? 1 : 0, 0, 0, c->stream));
        if (observe) CK(c, launch_cell_obs(d, 1, 1, c->stream));
    } else if (c->path == 1) {
        CK(c, launch_cell_build(d, c->stream));
        CK(c, launch_cell_density(d, observe ? 1 : 0, c->stream));
        CK(c, launch_cell_force(d, observe ? 1 : 0, 0, 0, c->stream));
        if (observe) CK(c, launch_cell_obs(d, 1, 1, c->stream));
    } else {
        CK(c, launch_density(d, i0, n0, c->shape[0], observe ? 1 : 0, c->stream));
        CK(c, launch_force(d, i1, n1, c->shape[1], observe ? 1 : 0, 0, 0, c->stream));
    }
    if (observe) CK(c, launch_obs_reduce(d, 0, 0, c->stream));
    return MD_OK;
}

md_status recompute_forces(md_ctx* c, bool new_origin) {
    if (new_origin) CK(c, launch_origin(c->dev, c->stream));
    md_status st = evaluate(c, false);
    if (st != MD_OK) return st;
    CK(c, cudaStreamSynchronize(c->stream));
    return MD_OK;
}

// Issue one chunk of M steps whose first step has global index s0 (only s0 mod obs_every matters).
md_status enqueue_chunk(md_ctx* c, int M, int64_t s0, int kind) {
    const Dev& d = c->dev;
    int n0, n1;
    const Item* i0 = items_for(c, c->shape[0], &n0);
    const Item* i1 = items_for(c, c->shape[1], &n1);
    const int oe = c->cfg.obs_every;
    if (kind == MD_LANGEVIN && c->cfg.precision == MD_PREC_MIXED) CK(c, launch_noise(d, M, c->stream));
    CK(c, launch_start(d, 0, c->stream));
    for (int k = 0; k < M; ++k) {
        const int64_t next = s0 + k + 1;
        const bool obs = oe > 0 && next % oe == 0;
        const bool last = k == M - 1;
        const int flags = (last ? 1 : 0) | (obs ? 2 : 0);
        if (c->path == 2) {
            // MIXED lists: within a chunk (not Berendsen) the previous force pass did the position kernel's work
            if (c->nqmax == 0 || k == 0 || kind == MD_BERENDSEN) CK(c, launch_v_pos(d, k, c->stream));
            CK(c, launch_cell_build(d, c->stream, 1, k, c->nqmax == 0));  // MIXED: the counts are already clear
            CK(c, launch_v_rebuild(d, 1, k, c->stream));
            CK(c, launch_v_density(d, obs ? 1 : 0, c->stream, k));
            CK(c, launch_v_force(d, 2, k, flags, c->stream));
            if (obs) CK(c, launch_cell_obs(d, kind == MD_BERENDSEN ? 1 : 0, kind == MD_BERENDSEN ? 0 : 1, c->stream));
            if (kind == MD_BERENDSEN) CK(c, launch_cell_ke(d, c->stream));
        } else if (c->path == 1) {
            CK(c, launch_cell_build(d, c->stream));
            CK(c, launch_cell_density(d, obs ? 1 : 0, c->stream));
            CK(c, launch_cell_force(d, 2, k, flags, c->stream));
            // Berendsen: positions now, velocities after the rescale (in k_berendsen)
            if (obs) CK(c, launch_cell_obs(d, kind == MD_BERENDSEN ? 1 : 0, kind == MD_BERENDSEN ? 0 : 1, c->stream));
            if (kind == MD_BERENDSEN) CK(c, launch_cell_ke(d, c->stream));
        } else {
            CK(c, launch_density(d, i0, n0, c->shape[0], obs ? 1 : 0, c->stream));
            CK(c, launch_force(d, i1, n1, c->shape[1], 2, k, flags, c->stream));
        }
        if (kind == MD_BERENDSEN) CK(c, launch_berendsen(d, k, last ? 1 : 0, c->stream));
        if (obs) CK(c, launch_obs_reduce(d, k, 1, c->stream));
    }
    CK(c, launch_advance(d, M, c->stream));
    return MD_OK;
}

md_status get_graph(md_ctx* c, int M, int64_t s0, int kind, cudaGraphExec_t* out) {
    GraphKey key{};
    key.M = M;
    key.obs_every = c->cfg.obs_every;
    key.phase = c->cfg.obs_every > 0 ? (int)(s0 % c->cfg.obs_every) : 0;
    key.kind = kind;
    key.dens[0] = c->shape[0].ipt;
    key.dens[1] = c->shape[0].warps;
    key.dens[2] = c->shape[0].cluster;
    key.force[0] = c->shape[1].ipt;
    key.force[1] = c->shape[1].warps;
    key.force[2] = c->shape[1].cluster;
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
        *out = it->second;
        return MD_OK;
    }
    if (c->graphs.size() >= 32) {
        for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
        c->graphs.clear();
    }
    cudaGraph_t g = nullptr;
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    md_status st = enqueue_chunk(c, M, s0, kind);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != MD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    CK(c, e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(c, e);
    c->graphs[key] = ex;
    *out = ex;
    return MD_OK;
}

void drop_graphs(md_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
    c->graphs.clear();
}

void free_all(md_ctx* c) {
    drop_graphs(c);
    void* ptrs[] = {c->d_poff, c->d_off, c->d_h_unit, c->d_h_ubase, c->d_h_pi, c->d_h_pj, c->d_nreal, c->d_clg,   c->d_status, c->d_x,      c->d_v,    c->d_mass,
                    c->d_rho,  c->d_origin, c->d_part, c->d_ke,     c->d_hist,   c->d_f,    c->d_mirror,
                    c->d_posg, c->d_step,  c->d_run,   c->items_d[0], c->items_d[1], c->items_d[2], c->d_hs, c->d_sig0, c->d_noise,
                    c->d_grid, c->d_cell_cl, c->d_cell_count, c->d_cell_atoms, c->d_eatom, c->d_obs_x, c->d_obs_v,
                    c->d_cpos, c->d_cposg, c->d_cell_order, c->d_cell_oct, c->d_cell_obyte,
                    c->d_vlist, c->d_vcount, c->d_vsub, c->d_vorder, c->d_vslotof, c->d_vslot, c->d_vhi,
                    c->d_q_n, c->d_cell_base, c->d_q_cell, c->d_q_list, c->d_q_count, c->d_q_ref, c->d_q_box,
                    c->d_vrcount, c->d_vrev, c->d_vrsub, c->d_hbuf, c->d_fbuf, c->d_rho_half, c->d_fhalf,
                    c->d_vcl, c->d_vcn, c->d_vflag,
                    c->d_vposg, c->d_vxref, c->d_vdmax,
                    c->sb.com, c->sb.core, c->sb.ncore, c->sb.hist, c->sb.ref, c->sb.ref_com, c->sb.sel, c->sb.msd,
                    c->sb.nsel, c->sb.nb, c->sb.nnb, c->sb.cls, c->sb.counts, c->sb.capped};
    for (void* p : ptrs) dfree(c, p);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->h_run) cudaFreeHost(c->h_run);
    if (c->h_step) cudaFreeHost(c->h_step);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

void fill_obs(const md_ctx* c, const double* h, int64_t step, double time_fs, md_obs* o) {
    o->epot_eV = h[0];
    o->ekin_eV = h[1];
    o->etot_eV = h[2];
    o->T_K = h[3];
    for (int k = 0; k < 3; ++k) {
        o->com_A[k] = h[4 + k];
        o->mom[k] = h[7 + k];
        o->angmom[k] = h[10 + k];
    }
    o->step = step;
    o->time_fs = time_fs;
    o->status = h[15] != 0.0 ? MD_ERR_NONFINITE : MD_OK;
    o->reserved = 0;
    (void)c;
}

md_status check_status(md_ctx* c) {
    int32_t s = 0;
    CK(c, cudaMemcpyAsync(&s, c->d_status, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (s & 1) return fail(c, MD_ERR_NONFINITE, "a force, position or velocity became non-finite");
    if (s & 2)
        return fail(c, MD_ERR_STATE, "a cell of the cell grid overflowed (more than %d atoms); forces are invalid",
                    kCellCap);
    if (s & 4)
        return fail(c, MD_ERR_STATE, "a neighbour list overflowed (more than %d entries); forces are invalid",
                    c->nqmax > 0 ? kQMax : kVMax);
    if (s & kStatusTimeout)
        return fail(c, MD_ERR_TIMEOUT, "a pair pass gave up waiting for its partial sums; forces are invalid");
    return MD_OK;
}

std::string tune_key(const md_ctx* c) {
    cudaDeviceProp p{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&p, dev);
    int maxn = 0;
    for (int s : c->sizes) maxn = std::max(maxn, s);
    char buf[512];
    snprintf(buf, sizeof buf, "%s|%d|prec%d|rc%g|B%d|N%lld|max%d", p.name, p.multiProcessorCount,
             c->cfg.precision, c->pot.rcut, c->B, (long long)c->ntot, maxn);
    std::string k = buf;
    for (char& ch : k)
        if (ch == '"' || ch == '\\') ch = '_';
    return k;
}

// Tiny JSON cache: {"key": [d_ipt, d_warps, d_cluster, f_ipt, f_warps, f_cluster], ...}
bool cache_lookup(const char* path, const std::string& key, Shape out[2]) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
    fclose(f);
    const std::string q = "\"" + key + "\"";
    size_t p = s.find(q);
    if (p == std::string::npos) return false;
    p = s.find('[', p);
    if (p == std::string::npos) return false;
    int v[6];
    if (sscanf(s.c_str() + p, "[%d,%d,%d,%d,%d,%d]", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) != 6) return false;
    Shape a{v[0], v[1], v[2]}, b{v[3], v[4], v[5]};
    if (!shape_ok(a, 0) || !shape_ok(b, 1)) return false;
    out[0] = a;
    out[1] = b;
    return true;
}

void cache_store(const char* path, const std::string& key, const Shape s[2]) {
    if (!path) return;
    std::map<std::string, std::string> entries;
    if (FILE* f = fopen(path, "r")) {
        std::string txt;
        char buf[4096];
        size_t n;
        while ((n = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, n);
        fclose(f);
        size_t p = 0;
        while ((p = txt.find('"', p)) != std::string::npos) {
            size_t e = txt.find('"', p + 1);
            if (e == std::string::npos) break;
            std::string k = txt.substr(p + 1, e - p - 1);
            size_t a = txt.find('[', e), b = txt.find(']', e);
            if (a == std::string::npos || b == std::string::npos) break;
            entries[k] = txt.substr(a, b - a + 1);
            p = b + 1;
        }
    }
    char val[128];
    snprintf(val, sizeof val, "[%d,%d,%d,%d,%d,%d]", s[0].ipt, s[0].warps, s[0].cluster, s[1].ipt, s[1].warps,
             s[1].cluster);
    entries[key] = val;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto& e : entries) fprintf(f, "  \"%s\": %s%s\n", e.first.c_str(), e.second.c_str(), ++k < entries.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

extern "C" {

int32_t md_abi_version(void) { return SCMD_ABI_VERSION; }

const char* md_last_error(const md_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

namespace {

// Pair path that md_create resolves from the configuration: 0 all pairs, 1 cells, 2 neighbour lists.
int resolve_path(const md_config* cfg, const md_sc_params* prm, int32_t n_clusters, const int32_t* sizes) {
    int maxn = 0;
    for (int b = 0; b < n_clusters; ++b) maxn = std::max(maxn, sizes[b]);
    // automatic: with a cutoff and a large cluster (or a shifted cutoff), the neighbour lists (quad
    // lists in MIXED, per-atom lists in FP64)
    const bool big = cfg->path == MD_PATH_AUTO && prm->rcut_A > 0 && (maxn >= kAutoCellsMinAtoms || prm->cutoff_shift);
    const bool verlet = cfg->path == MD_PATH_VERLET || big;
    const bool cells = verlet || cfg->path == MD_PATH_CELLS;
    return verlet ? 2 : (cells ? 1 : 0);
}

// md_create (host arrays) and md_create_device on the all-pairs path (device arrays: on_device;
// the values are then validated on the GPU before they are used).
md_status create_impl(const md_config* cfg, int32_t n_clusters, const int32_t* sizes, const double* pos,
                      const double* vel, const double* mass, bool on_device, const md_sc_params* prm, md_ctx** out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, MD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!cfg || !sizes || !pos || !mass || !prm) return fail(nullptr, MD_ERR_INVALID, "NULL argument");
    if (n_clusters < 1) return fail(nullptr, MD_ERR_INVALID, "n_clusters must be >= 1");
    if (cfg->precision != MD_PREC_FP64 && cfg->precision != MD_PREC_MIXED)
        return fail(nullptr, MD_ERR_INVALID, "unknown precision %d", cfg->precision);
    if (cfg->path != MD_PATH_AUTO && cfg->path != MD_PATH_ALLPAIRS && cfg->path != MD_PATH_CELLS &&
        cfg->path != MD_PATH_VERLET && cfg->path != MD_PATH_ALLPAIRS_HALF)
        return fail(nullptr, MD_ERR_INVALID, "unknown path %d", cfg->path);
    if (cfg->path == MD_PATH_ALLPAIRS_HALF && cfg->precision != MD_PREC_FP64)
        return fail(nullptr, MD_ERR_INVALID, "MD_PATH_ALLPAIRS_HALF runs in FP64 only");
    if ((cfg->path == MD_PATH_CELLS || cfg->path == MD_PATH_VERLET) && !(prm->rcut_A > 0))
        return fail(nullptr, MD_ERR_INVALID, "the cell and neighbour-list paths need a cutoff (rcut_A > 0)");
    if (cfg->obs_every < 0 || cfg->graph_chunk < 0 || cfg->obs_capacity < 0)
        return fail(nullptr, MD_ERR_INVALID, "negative obs_every, graph_chunk or obs_capacity");
    if (!(std::isfinite(prm->eps_eV) && std::isfinite(prm->c) && std::isfinite(prm->a_A) && prm->a_A > 0 &&
          std::isfinite(prm->rcut_A) && prm->rcut_A >= 0 && prm->n >= 1 && prm->n <= 32 && prm->m >= 1 &&
          prm->m <= 32 && (prm->cutoff_shift == 0 || prm->cutoff_shift == 1) && prm->reserved == 0))
        return fail(nullptr, MD_ERR_INVALID, "invalid Sutton-Chen parameters");
    if (prm->cutoff_shift && !(prm->rcut_A > 0))
        return fail(nullptr, MD_ERR_INVALID, "a shifted cutoff needs rcut_A > 0");
    if (prm->cutoff_shift && (cfg->path == MD_PATH_ALLPAIRS || cfg->path == MD_PATH_ALLPAIRS_HALF))
        return fail(nullptr, MD_ERR_INVALID, "the shifted cutoff runs on the cell and neighbour-list paths");
    int64_t ntot = 0;
    for (int b = 0; b < n_clusters; ++b) {
        if (sizes[b] < 1) return fail(nullptr, MD_ERR_INVALID, "cluster %d has size %d", b, sizes[b]);
        ntot += sizes[b];
    }
    if (ntot > 200000000) return fail(nullptr, MD_ERR_INVALID, "too many atoms");
    if (!on_device) {
        if (!finite_all(pos, 3 * ntot)) return fail(nullptr, MD_ERR_INVALID, "non-finite position");
        if (vel && !finite_all(vel, 3 * ntot)) return fail(nullptr, MD_ERR_INVALID, "non-finite velocity");
        for (int64_t k = 0; k < ntot; ++k)
            if (!(std::isfinite(mass[k]) && mass[k] > 0))
                return fail(nullptr, MD_ERR_INVALID, "mass %lld invalid", (long long)k);
    }

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1)
        return fail(nullptr, MD_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    if (prop.major < 10) return fail(nullptr, MD_ERR_CUDA, "device %s (sm_%d%d) is not an sm_103a part", prop.name, prop.major, prop.minor);

    md_ctx* c = new md_ctx();
    c->cfg = *cfg;
    if (c->cfg.graph_chunk == 0) c->cfg.graph_chunk = 256;
    c->hist_cap = cfg->obs_capacity > 0 ? cfg->obs_capacity : 4096;
    c->B = n_clusters;
    c->ntot = ntot;
    c->sizes.assign(sizes, sizes + n_clusters);
    c->off.resize(n_clusters + 1);
    c->poff.resize(n_clusters + 1);
    c->off[0] = c->poff[0] = 0;
    for (int b = 0; b < n_clusters; ++b) {
        c->off[b + 1] = c->off[b] + sizes[b];
        c->poff[b + 1] = c->poff[b] + ((sizes[b] + kPad - 1) / kPad) * kPad;
    }
    c->npad = c->poff[n_clusters];
    c->ngroups = c->npad / kGroup;
    c->cl_of_group.resize(c->ngroups);
    for (int b = 0; b < n_clusters; ++b)
        for (int g = c->poff[b] / kGroup; g < c->poff[b + 1] / kGroup; ++g) c->cl_of_group[g] = b;
    for (int k = 0; k < 3; ++k) {
        const int BI = 32 << k;
        for (int b = 0; b < n_clusters; ++b)
            for (int a = 0; a < sizes[b]; a += BI) {
                Item it{};
                it.i0 = c->poff[b] + a;
                it.ni = std::min(BI, sizes[b] - a);
                it.j0 = c->poff[b];
                it.nj = sizes[b];
                it.cl = b;
                c->items_h[k].push_back(it);
            }
        // largest clusters first: long items start early, short ones fill the tail
        std::stable_sort(c->items_h[k].begin(), c->items_h[k].end(),
                         [](const Item& x, const Item& y) { return x.nj > y.nj; });
    }
    // potential constants
    Pot& P = c->pot;
    P.eps = prm->eps_eV;
    P.c = prm->c;
    P.a = prm->a_A;
    P.n = prm->n;
    P.m = prm->m;
    P.rcut = prm->rcut_A;
    P.rcut2 = prm->rcut_A > 0 ? prm->rcut_A * prm->rcut_A : 0.0;
    P.A9 = P.eps * P.n * std::pow(P.a, P.n);
    P.B6 = P.eps * P.c * P.m * 0.5 * std::pow(P.a, P.m);
    P.am = std::pow(P.a, P.m);
    P.ecoef = 0.5 * P.eps * std::pow(P.a, P.n);
    P.A9f = (float)P.A9;
    P.rcut2f = (float)P.rcut2;
    P.gsf = (float)(P.B6 / std::sqrt(P.am));
    P.special = (P.n == 9 && P.m == 6) ? 1 : 0;
    P.shift = prm->cutoff_shift;
    P.shm = P.shift ? std::pow(P.rcut, -(double)P.m) : 0.0;
    P.shn = P.shift ? std::pow(P.rcut, -(double)P.n) : 0.0;
    {
        c->path = resolve_path(cfg, prm, n_clusters, sizes);
        const bool cells = c->path >= 1;
        if (cells && on_device) {  // md_create_device reads the positions back for the cell grids first
            delete c;
            return fail(nullptr, MD_ERR_INVALID, "internal: device positions on a cell path");
        }
        // FP64 lists address a pair's place in 32 bits: nslot * kVMax < 2^32
        const int64_t vmax_atoms = cfg->precision == MD_PREC_FP64 ? (1 << 23) : (1 << 26);
        if (c->path == 2 && c->ntot >= vmax_atoms) {
            delete c;
            return fail(nullptr, MD_ERR_INVALID, "the neighbour-list path takes fewer than %lld atoms in this precision",
                        (long long)vmax_atoms);
        }
        // the neighbour lists hold the pairs within rcut + skin, so their cells are sized by that
        if (cells && !make_grids(c, pos, mass, c->path == 2 ? P.rcut + kSkin : P.rcut)) {
            delete c;
            return fail(nullptr, MD_ERR_INVALID,
                        "rcut_A = %g is too large for the cell path (a cell would exceed %d atoms); "
                        "use MD_PATH_ALLPAIRS", P.rcut, kCellCap);
        }
    }

    auto bail = [&](md_status st) {
        free_all(c);
        g_create_error = c->err;
        delete c;
        return st;
    };
#define CKC(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            fail(c, e_ == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA, "%s failed: %s", #call, \
                 cudaGetErrorString(e_));                                                          \
            return bail(e_ == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA);               \
        }                                                                                          \
    } while (0)

    if (cfg->stream) {
        c->stream = reinterpret_cast<cudaStream_t>(cfg->stream);
    } else {
        CKC(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    CKC(configure_kernels());
    const size_t np = c->npad;
    CKC(dmalloc(c, &c->d_poff, sizeof(int32_t) * (n_clusters + 1)));
    CKC(dmalloc(c, &c->d_off, sizeof(int32_t) * (n_clusters + 1)));
    CKC(dmalloc(c, &c->d_nreal, sizeof(int32_t) * n_clusters));
    CKC(dmalloc(c, &c->d_clg, sizeof(int32_t) * c->ngroups));
    CKC(dmalloc(c, &c->d_status, sizeof(int32_t)));
    CKC(dmalloc(c, &c->d_x, sizeof(double) * 3 * np));
    CKC(dmalloc(c, &c->d_v, sizeof(double) * 3 * np));
    CKC(dmalloc(c, &c->d_mass, sizeof(double) * np));
    CKC(dmalloc(c, &c->d_rho, sizeof(double) * np));
    CKC(dmalloc(c, &c->d_origin, sizeof(double) * 3 * n_clusters));
    CKC(dmalloc(c, &c->d_hs, sizeof(double) * np));
    CKC(dmalloc(c, &c->d_sig0, sizeof(float) * np));
    if (cfg->precision == MD_PREC_MIXED) {
        // Langevin normals of a whole chunk are drawn ahead of it; the buffer holds at most
        // 256 MB, which bounds the chunk length for very large batches.
        const size_t per_step = sizeof(float4) * np;
        c->noise_steps = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->cfg.graph_chunk, (256u << 20) / per_step));
        CKC(dmalloc(c, &c->d_noise, per_step * c->noise_steps));
    }
    CKC(dmalloc(c, &c->d_part, sizeof(double) * kObsFields * c->ngroups));
    CKC(dmalloc(c, &c->d_ke, sizeof(double) * c->ngroups));
    CKC(dmalloc(c, &c->d_hist, sizeof(double) * kHistFields * (size_t)n_clusters * (c->hist_cap + 1)));
    CKC(dmalloc(c, &c->d_f, (size_t)elem_size(c) * 3 * np));
    CKC(dmalloc(c, &c->d_mirror, (size_t)vec4_size(c) * np));
    CKC(dmalloc(c, &c->d_posg, (size_t)vec4_size(c) * np));
    CKC(dmalloc(c, &c->d_step, sizeof(int64_t)));
    CKC(dmalloc(c, &c->d_run, sizeof(Run)));
    if (c->path >= 1) {
        std::vector<int32_t> cell_cl(c->n_cells), order(c->n_cells);
        std::vector<double> depth(c->n_cells);
        for (int b = 0; b < n_clusters; ++b) {
            const CellGrid& g = c->grids[b];
            for (int k = 0; k < g.G * g.G * g.G; ++k) {
                cell_cl[g.off + k] = b;
                // distance of the cell centre from the grid centre, in units of the cluster radius
                const double x = (k % g.G + 0.5) * g.h - g.E, y = ((k / g.G) % g.G + 0.5) * g.h - g.E;
                const double z = (k / (g.G * g.G) + 0.5) * g.h - g.E;
                depth[g.off + k] = std::sqrt(x * x + y * y + z * z) / std::max(g.E - c->pot.rcut, 1e-9);
            }
        }
        // interior (fullest) cells are launched first, so that the light surface cells and the empty
        // ones fill the tail of the pass instead of extending it
        for (int k = 0; k < c->n_cells; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return depth[a] < depth[b]; });
        CKC(dmalloc(c, &c->d_grid, sizeof(CellGrid) * n_clusters));
        CKC(dmalloc(c, &c->d_cell_cl, sizeof(int32_t) * c->n_cells));
        CKC(dmalloc(c, &c->d_cell_order, sizeof(int32_t) * c->n_cells));
        CKC(cudaMemcpyAsync(c->d_cell_order, order.data(), sizeof(int32_t) * c->n_cells, cudaMemcpyHostToDevice, c->stream));
        CKC(dmalloc(c, &c->d_cell_count, sizeof(int32_t) * c->n_cells));
        CKC(dmalloc(c, &c->d_cell_atoms, sizeof(int32_t) * kCellCap * (size_t)c->n_cells));
        CKC(dmalloc(c, &c->d_cell_oct, sizeof(int32_t) * 9 * (size_t)c->n_cells));
        CKC(dmalloc(c, &c->d_cell_obyte, (size_t)kCellCap * c->n_cells));
        CKC(cudaMemsetAsync(c->d_cell_oct, 0, sizeof(int32_t) * 9 * (size_t)c->n_cells, c->stream));
        CKC(dmalloc(c, &c->d_cpos, (size_t)vec4_size(c) * kCellCap * c->n_cells));
        CKC(dmalloc(c, &c->d_cposg, (size_t)vec4_size(c) * kCellCap * c->n_cells));
        CKC(dmalloc(c, &c->d_eatom, sizeof(double) * 2 * np));
        CKC(dmalloc(c, &c->d_obs_x, sizeof(double) * 3 * np));
        CKC(dmalloc(c, &c->d_obs_v, sizeof(double) * 3 * np));
        CKC(cudaMemcpyAsync(c->d_grid, c->grids.data(), sizeof(CellGrid) * n_clusters, cudaMemcpyHostToDevice, c->stream));
        CKC(cudaMemcpyAsync(c->d_cell_cl, cell_cl.data(), sizeof(int32_t) * c->n_cells, cudaMemcpyHostToDevice, c->stream));
        CKC(cudaMemsetAsync(c->d_cell_count, 0, sizeof(int32_t) * c->n_cells, c->stream));
        CKC(cudaMemsetAsync(c->d_eatom, 0, sizeof(double) * 2 * np, c->stream));
        CKC(cudaMemsetAsync(c->d_obs_x, 0, sizeof(double) * 3 * np, c->stream));
        CKC(cudaMemsetAsync(c->d_obs_v, 0, sizeof(double) * 3 * np, c->stream));
    }
    if (c->path == 2) {
        const bool quads = cfg->precision == MD_PREC_MIXED;
        // MIXED: every cell's atoms padded to whole quads (at most 3 empty slots per cell)
        c->nqmax = quads ? (int)((c->ntot + 3 * (int64_t)c->n_cells + 3) / 4) : 0;
        const size_t ns = quads ? 4 * (size_t)c->nqmax : (size_t)c->ntot;
        c->nslot = (int32_t)ns;
        CKC(dmalloc(c, &c->d_vorder, sizeof(int32_t) * ns));
        CKC(dmalloc(c, &c->d_vslotof, sizeof(int32_t) * np));
        // MIXED: 4 more slots for the padding quad of the lists (index nqmax), far from every atom
        const size_t ns_alloc = quads ? ns + 4 : ns;
        CKC(dmalloc(c, &c->d_vhi, (size_t)vec4_size(c) * ns_alloc));
        // MIXED: the force pass reads a 32-byte record per slot, the offset and g (float4) then its quad's
        // reference point (float4)
        CKC(dmalloc(c, &c->d_vposg, (quads ? 2 * sizeof(float4) : (size_t)vec4_size(c)) * ns_alloc));
        CKC(dmalloc(c, &c->d_vxref, sizeof(double) * 3 * ns));
        CKC(dmalloc(c, &c->d_vdmax, sizeof(uint32_t) * 2));
        CKC(cudaMemsetAsync(c->d_vdmax, 0, sizeof(uint32_t) * 2, c->stream));
        // every slot and entry starts as a valid index (atom 0, empty list)
        CKC(cudaMemsetAsync(c->d_vorder, 0, sizeof(int32_t) * ns, c->stream));
        CKC(cudaMemsetAsync(c->d_vslotof, 0, sizeof(int32_t) * np, c->stream));
        CKC(cudaMemsetAsync(c->d_vxref, 0, sizeof(double) * 3 * ns, c->stream));
        if (quads) {
            const size_t nq = (size_t)c->nqmax;
            CKC(dmalloc(c, &c->d_q_n, sizeof(int32_t)));
            CKC(dmalloc(c, &c->d_cell_base, sizeof(int32_t) * (c->n_cells + 1)));
            CKC(dmalloc(c, &c->d_q_ref, sizeof(float4) * (nq + 1)));
            CKC(dmalloc(c, &c->d_q_box, sizeof(float4) * 2 * nq));
            CKC(dmalloc(c, &c->d_q_cell, sizeof(int32_t) * nq));
            CKC(dmalloc(c, &c->d_q_list, sizeof(int32_t) * kQMax * nq));
            CKC(dmalloc(c, &c->d_q_count, sizeof(int32_t) * nq));
            CKC(cudaMemsetAsync(c->d_q_n, 0, sizeof(int32_t), c->stream));
            CKC(cudaMemsetAsync(c->d_cell_base, 0, sizeof(int32_t) * (c->n_cells + 1), c->stream));
            CKC(cudaMemsetAsync(c->d_q_count, 0, sizeof(int32_t) * nq, c->stream));
            {  // the padding quad of the lists: reference point 0, its 4 slots far from every atom and every
               // empty slot (g = 0)
                constexpr float F = -kQuadFar;
                static const float far4[4][4] = {{F, F, F, 0.f}, {F, F, F, 0.f}, {F, F, F, 0.f}, {F, F, F, 0.f}};
                static const float far8[8][4] = {{F, F, F, 0.f}, {0.f, 0.f, 0.f, 0.f}, {F, F, F, 0.f}, {0.f, 0.f, 0.f, 0.f},
                                                 {F, F, F, 0.f}, {0.f, 0.f, 0.f, 0.f}, {F, F, F, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                CKC(cudaMemcpyAsync(static_cast<float4*>(c->d_vhi) + ns, far4, sizeof far4, cudaMemcpyHostToDevice,
                                    c->stream));
                CKC(cudaMemcpyAsync(static_cast<float4*>(c->d_vposg) + 2 * ns, far8, sizeof far8,
                                    cudaMemcpyHostToDevice, c->stream));
                CKC(cudaMemsetAsync(c->d_q_ref + nq, 0, sizeof(float4), c->stream));
            }
        } else {
            CKC(dmalloc(c, &c->d_vlist, sizeof(int32_t) * kVMax * ns));
            CKC(dmalloc(c, &c->d_vcount, sizeof(int32_t) * ns));
            CKC(dmalloc(c, &c->d_vsub, sizeof(int32_t) * kVLanes * ns));
            CKC(dmalloc(c, &c->d_vslot, sizeof(int32_t)));
            CKC(dmalloc(c, &c->d_vrcount, sizeof(int32_t) * ns));
            CKC(dmalloc(c, &c->d_vrev, sizeof(uint64_t) * kVMax * ns));
            CKC(dmalloc(c, &c->d_vrsub, sizeof(int32_t) * kVLanes * ns));
            CKC(dmalloc(c, &c->d_vcl, sizeof(int2) * kVMax * ns));
            CKC(dmalloc(c, &c->d_vcn, sizeof(int32_t) * ns));
            CKC(dmalloc(c, &c->d_vflag, (size_t)kVMax * ns));
            CKC(cudaMemsetAsync(c->d_vflag, 0, (size_t)kVMax * ns, c->stream));
            CKC(cudaMemsetAsync(c->d_vrsub, 0, sizeof(int32_t) * kVLanes * ns, c->stream));
            CKC(dmalloc(c, &c->d_hbuf, sizeof(double) * kVMax * ns));
            CKC(dmalloc(c, &c->d_fbuf, sizeof(double4) * kVMax * ns));
            CKC(dmalloc(c, &c->d_rho_half, sizeof(double) * ns));
            CKC(dmalloc(c, &c->d_fhalf, sizeof(double4) * ns));
            CKC(cudaMemsetAsync(c->d_vrcount, 0, sizeof(int32_t) * ns, c->stream));
            CKC(cudaMemsetAsync(c->d_vlist, 0, sizeof(int32_t) * kVMax * ns, c->stream));
            CKC(cudaMemsetAsync(c->d_vcount, 0, sizeof(int32_t) * ns, c->stream));
            CKC(cudaMemsetAsync(c->d_vsub, 0, sizeof(int32_t) * kVLanes * ns, c->stream));
        }
    }
    {
        // FP64 all pairs: the work units of the each-pair-once kernels, when that form is chosen
        std::vector<int4> units;
        std::vector<int32_t> ubase(n_clusters);
        if (c->path == 0 && cfg->precision == MD_PREC_FP64 &&
            (cfg->path == MD_PATH_AUTO || cfg->path == MD_PATH_ALLPAIRS_HALF)) {
            for (int b = 0; b < n_clusters; ++b) {
                ubase[b] = (int32_t)units.size();
                const int n = sizes[b], T = (n + 31) / 32, H = (n + 15) / 16;
                for (int I = 0; I < T; ++I)
                    for (int h = 2 * I; h < H; ++h)
                        units.push_back(make_int4(c->poff[b] + 32 * I, c->poff[b] + 16 * h, h < 2 * I + 2 ? 1 : 0, b));
            }
            // pair-weighted mean cluster size sum n^3 / sum n^2: small clusters waste much of a unit
            double s2 = 0.0, s3 = 0.0;
            for (int b = 0; b < n_clusters; ++b) {
                s2 += (double)sizes[b] * sizes[b];
                s3 += (double)sizes[b] * sizes[b] * sizes[b];
            }
            c->half = cfg->path == MD_PATH_ALLPAIRS_HALF ||
                      (units.size() >= (size_t)kHalfMinUnits && s3 >= kHalfMinMeanSize * s2);
        }
        if (c->half) {
            c->h_nunits = (int32_t)units.size();
            CKC(dmalloc(c, &c->d_h_unit, sizeof(int4) * units.size()));
            CKC(dmalloc(c, &c->d_h_ubase, sizeof(int32_t) * n_clusters));
            CKC(dmalloc(c, &c->d_h_pi, (size_t)32 * 32 * units.size()));
            CKC(dmalloc(c, &c->d_h_pj, (size_t)16 * 32 * units.size()));
            CKC(cudaMemcpyAsync(c->d_h_unit, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice, c->stream));
            CKC(cudaMemcpyAsync(c->d_h_ubase, ubase.data(), sizeof(int32_t) * n_clusters, cudaMemcpyHostToDevice,
                                c->stream));
        }
    }
    for (int k = 0; k < 3; ++k) {
        CKC(dmalloc(c, &c->items_d[k], sizeof(Item) * std::max<size_t>(1, c->items_h[k].size())));
        CKC(cudaMemcpyAsync(c->items_d[k], c->items_h[k].data(), sizeof(Item) * c->items_h[k].size(), cudaMemcpyHostToDevice, c->stream));
    }
    c->h_stage_n = std::max<size_t>(6 * np, 16);
    CKC(cudaMallocHost(&c->h_stage, sizeof(double) * c->h_stage_n));
    CKC(cudaMallocHost(&c->h_run, sizeof(Run)));
    CKC(cudaMallocHost(&c->h_step, sizeof(int64_t)));
    std::vector<int32_t> nreal(sizes, sizes + n_clusters);
    CKC(cudaMemcpyAsync(c->d_poff, c->poff.data(), sizeof(int32_t) * (n_clusters + 1), cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->d_off, c->off.data(), sizeof(int32_t) * (n_clusters + 1), cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->d_nreal, nreal.data(), sizeof(int32_t) * n_clusters, cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->d_clg, c->cl_of_group.data(), sizeof(int32_t) * c->ngroups, cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream));
    CKC(cudaMemsetAsync(c->d_part, 0, sizeof(double) * kObsFields * c->ngroups, c->stream));
    CKC(cudaMemsetAsync(c->d_ke, 0, sizeof(double) * c->ngroups, c->stream));
    CKC(cudaMemsetAsync(c->d_hist, 0, sizeof(double) * kHistFields * (size_t)n_clusters * (c->hist_cap + 1), c->stream));
    CKC(cudaMemsetAsync(c->d_f, 0, (size_t)elem_size(c) * 3 * np, c->stream));
    CKC(cudaMemsetAsync(c->d_rho, 0, sizeof(double) * np, c->stream));
    CKC(cudaMemsetAsync(c->d_step, 0, sizeof(int64_t), c->stream));
    // masses (padding atoms get mass 1 so that no division by zero can occur; device input: k_import)
    if (!on_device) {
        std::vector<double> m(np, 1.0);
        for (int b = 0; b < n_clusters; ++b)
            for (int a = 0; a < sizes[b]; ++a) m[c->poff[b] + a] = mass[c->off[b] + a];
        CKC(cudaMemcpyAsync(c->d_mass, m.data(), sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
    }
    // padding atoms of the mirror and posg buffers: far apart and far from everything, g = 0
    {
        const bool mixed = cfg->precision == MD_PREC_MIXED;
        std::vector<unsigned char> pad((size_t)vec4_size(c) * np, 0);
        for (int b = 0; b < n_clusters; ++b)
            for (int a = sizes[b]; a < c->poff[b + 1] - c->poff[b]; ++a) {
                const size_t p = c->poff[b] + a;
                const double far = (mixed ? 1.0e18 : 1.0e150) * (1.0 + (a - sizes[b]));
                if (mixed) {
                    float v[4] = {(float)far, 0.f, 0.f, 0.f};
                    memcpy(pad.data() + 16 * p, v, 16);
                } else {
                    double v[4] = {far, 0.0, 0.0, 0.0};
                    memcpy(pad.data() + 32 * p, v, 32);
                }
            }
        CKC(cudaMemcpyAsync(c->d_mirror, pad.data(), pad.size(), cudaMemcpyHostToDevice, c->stream));
        CKC(cudaMemcpyAsync(c->d_posg, pad.data(), pad.size(), cudaMemcpyHostToDevice, c->stream));
    }
    fill_dev(c);
    c->shape[0] = default_shape(c, 0);
    c->shape[1] = default_shape(c, 1);
    {
        Shape cached[2];
        if (cfg->tune_cache && cache_lookup(cfg->tune_cache, tune_key(c), cached)) {
            c->shape[0] = cached[0];
            c->shape[1] = cached[1];
        }
    }
    md_status st = MD_OK;
    if (on_device) {
        CKC(launch_check_input(pos, vel, mass, ntot, c->d_status, c->stream));
        int32_t flag = 0;
        CKC(cudaMemcpyAsync(&flag, c->d_status, sizeof flag, cudaMemcpyDeviceToHost, c->stream));
        CKC(cudaStreamSynchronize(c->stream));
        if (flag & invalid_input_bit()) {
            fail(c, MD_ERR_INVALID, "non-finite position or velocity, or a mass that is not finite and > 0");
            return bail(MD_ERR_INVALID);
        }
        CKC(launch_import(c->dev, c->d_off, pos, vel, mass, c->stream));
    } else {
        st = upload_state(c, pos, vel);
    }
    if (st != MD_OK) return bail(st);
    // Run parameters used by the observable reduction before the first md_step
    memset(c->h_run, 0, sizeof(Run));
    c->h_run->kb = kKB;
    c->h_run->nsteps = 1;
    c->h_run->hist_cap = c->hist_cap;
    c->h_run->obs_every = c->cfg.obs_every;
    CKC(cudaMemcpyAsync(c->d_run, c->h_run, sizeof(Run), cudaMemcpyHostToDevice, c->stream));
    st = recompute_forces(c, true);
    if (st == MD_OK) st = check_status(c);
    if (st != MD_OK) return bail(st);
    if (cfg->tune == 1) {
        st = md_autotune(c, 10);
        if (st != MD_OK) return bail(st);
    }
#undef CKC
    *out = c;
    return MD_OK;
}

}  // namespace

extern "C" {

md_status md_create(const md_config* cfg, int32_t n_clusters, const int32_t* sizes, const double* pos,
                    const double* vel, const double* mass, const md_sc_params* prm, md_ctx** out) {
    return create_impl(cfg, n_clusters, sizes, pos, vel, mass, false, prm, out);
}

md_status md_create_device(const md_config* cfg, int32_t n_clusters, const int32_t* sizes, const double* pos_dev,
                           const double* vel_dev, const double* mass_dev, const md_sc_params* prm, md_ctx** out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, MD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!cfg || !sizes || !pos_dev || !mass_dev || !prm) return fail(nullptr, MD_ERR_INVALID, "NULL argument");
    if (n_clusters < 1) return fail(nullptr, MD_ERR_INVALID, "n_clusters must be >= 1");
    int64_t ntot = 0;
    for (int b = 0; b < n_clusters; ++b) {
        if (sizes[b] < 1) return fail(nullptr, MD_ERR_INVALID, "cluster %d has size %d", b, sizes[b]);
        ntot += sizes[b];
    }
    if (ntot > 200000000) return fail(nullptr, MD_ERR_INVALID, "too many atoms");
    if (resolve_path(cfg, prm, n_clusters, sizes) == 0)
        return create_impl(cfg, n_clusters, sizes, pos_dev, vel_dev, mass_dev, true, prm, out);
    // The cell and neighbour-list paths size each cluster's grid from its positions on the host:
    // the three arrays are read back once, on the given stream, and the context is made from them.
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cfg->stream);
    std::vector<double> p(3 * (size_t)ntot), v(vel_dev ? 3 * (size_t)ntot : 0), m((size_t)ntot);
    cudaError_t e = cudaMemcpyAsync(p.data(), pos_dev, sizeof(double) * p.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && vel_dev)
        e = cudaMemcpyAsync(v.data(), vel_dev, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.data(), mass_dev, sizeof(double) * m.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return fail(nullptr, MD_ERR_CUDA, "reading the device arrays failed: %s", cudaGetErrorString(e));
    return create_impl(cfg, n_clusters, sizes, p.data(), vel_dev ? v.data() : nullptr, m.data(), false, prm, out);
}

void md_destroy(md_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

md_status md_energy_forces(md_ctx* c, double* epot, double* forces) {
    if (!c) return MD_ERR_INVALID;
    md_status st = evaluate(c, true);
    if (st != MD_OK) return st;
    if (epot) {
        double* h = c->h_stage;
        CK(c, cudaMemcpyAsync(h, c->d_hist + (size_t)c->hist_cap * c->B * kHistFields,
                              sizeof(double) * kHistFields * c->B, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        for (int b = 0; b < c->B; ++b) epot[b] = h[(size_t)b * kHistFields];
    }
    if (forces) {
        st = md_get_forces(c, forces);
        if (st != MD_OK) return st;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return check_status(c);
}

md_status md_get_forces(md_ctx* c, double* forces) {
    if (!c || !forces) return MD_ERR_INVALID;
    double* st = c->h_stage;
    if (c->cfg.precision == MD_PREC_MIXED) {
        float* tmp = reinterpret_cast<float*>(st + 3 * (size_t)c->npad);
        CK(c, cudaMemcpyAsync(tmp, c->d_f, sizeof(float) * 3 * c->npad, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        for (size_t k = 0; k < 3 * (size_t)c->npad; ++k) st[k] = tmp[k];
    } else {
        CK(c, cudaMemcpyAsync(st, c->d_f, sizeof(double) * 3 * c->npad, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    unpack(c, st, forces);
    return MD_OK;
}

md_status md_get_density(md_ctx* c, double* rho) {
    if (!c || !rho) return MD_ERR_INVALID;
    double* st = c->h_stage;
    CK(c, cudaMemcpyAsync(st, c->d_rho, sizeof(double) * c->npad, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int b = 0; b < c->B; ++b)
        for (int a = 0; a < c->sizes[b]; ++a) rho[c->off[b] + a] = st[c->poff[b] + a];
    return MD_OK;
}

md_status md_step(md_ctx* c, int64_t nsteps, double dt, const md_thermostat* th) {
    if (!c) return MD_ERR_INVALID;
    if (nsteps < 0) return fail(c, MD_ERR_INVALID, "nsteps < 0");
    if (nsteps == 0) return MD_OK;
    if (!(std::isfinite(dt) && dt > 0)) return fail(c, MD_ERR_INVALID, "dt must be finite and > 0");
    md_thermostat nve{};
    nve.kind = MD_NVE;
    const md_thermostat& t = th ? *th : nve;
    if (t.kind != MD_NVE && t.kind != MD_LANGEVIN && t.kind != MD_BERENDSEN)
        return fail(c, MD_ERR_INVALID, "unknown thermostat kind %d", t.kind);
    if (t.kind != MD_NVE && !(std::isfinite(t.T0_K) && std::isfinite(t.T1_K) && t.T0_K >= 0 && t.T1_K >= 0))
        return fail(c, MD_ERR_INVALID, "invalid target temperatures");
    if (t.kind == MD_LANGEVIN && !(std::isfinite(t.gamma_per_ps) && t.gamma_per_ps >= 0))
        return fail(c, MD_ERR_INVALID, "invalid Langevin friction");
    if (t.kind == MD_BERENDSEN && !(std::isfinite(t.tau_ps) && t.tau_ps * 1e3 > dt))
        return fail(c, MD_ERR_INVALID, "Berendsen tau must exceed dt");
    Run& r = *c->h_run;
    memset(&r, 0, sizeof r);
    r.dt = dt;
    r.h = 0.5 * dt;
    r.c1 = t.kind == MD_LANGEVIN ? std::exp(-t.gamma_per_ps * 1e-3 * dt) : 1.0;
    r.hk = r.h * (1.0 + r.c1);
    r.noise_k = t.kind == MD_LANGEVIN ? (1.0 - r.c1 * r.c1) * kKB * kConv : 0.0;
    r.T0 = t.T0_K;
    r.T1 = t.T1_K;
    r.dT = (t.T1_K - t.T0_K) / (double)nsteps;
    r.dt_over_tau = t.kind == MD_BERENDSEN ? dt / (t.tau_ps * 1e3) : 0.0;
    r.kb = kKB;
    r.step0 = c->step;
    r.nsteps = nsteps;
    r.seed = t.seed;
    r.kind = t.kind;
    r.obs_every = c->cfg.obs_every;
    r.hist_cap = c->hist_cap;
    CK(c, cudaMemcpyAsync(c->d_run, c->h_run, sizeof(Run), cudaMemcpyHostToDevice, c->stream));
    CK(c, launch_prepare(c->dev, c->stream));
    md_status st = set_step_base(c, c->step);
    if (st != MD_OK) return st;
    const int chunk = c->cfg.precision == MD_PREC_MIXED ? std::min(c->cfg.graph_chunk, c->noise_steps)
                                                        : c->cfg.graph_chunk;
    int64_t done = 0;
    const double t_call0 = c->time_fs;
    while (done < nsteps) {
        const int M = (int)std::min<int64_t>(chunk, nsteps - done);
        cudaGraphExec_t ex = nullptr;
        st = get_graph(c, M, c->step + done, t.kind, &ex);
        if (st != MD_OK) return st;
        CK(c, cudaGraphLaunch(ex, c->stream));
        done += M;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    // bookkeeping of recorded samples
    const int oe = c->cfg.obs_every;
    if (oe > 0) {
        for (int64_t s = ((c->step / oe) + 1) * oe; s <= c->step + nsteps; s += oe) {
            c->samples.emplace_back(s, t_call0 + (double)(s - c->step) * dt);
            if ((int)c->samples.size() > c->hist_cap) c->samples.pop_front();
        }
    }
    c->step += nsteps;
    c->time_fs = t_call0 + (double)nsteps * dt;
    return check_status(c);
}

md_status md_observables(md_ctx* c, md_obs* out) {
    if (!c || !out) return MD_ERR_INVALID;
    md_status st = evaluate(c, true);
    if (st != MD_OK) return st;
    double* h = c->h_stage;
    CK(c, cudaMemcpyAsync(h, c->d_hist + (size_t)c->hist_cap * c->B * kHistFields, sizeof(double) * kHistFields * c->B,
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int b = 0; b < c->B; ++b) fill_obs(c, h + (size_t)b * kHistFields, c->step, c->time_fs, out + b);
    return check_status(c);
}

md_status md_obs_history(md_ctx* c, md_obs* out, int32_t max_samples, int32_t* n_samples) {
    if (!c || !n_samples || (max_samples > 0 && !out)) return MD_ERR_INVALID;
    const int n = std::min<int>((int)c->samples.size(), std::max(0, max_samples));
    *n_samples = n;
    if (n == 0) return MD_OK;
    std::vector<double> h((size_t)kHistFields * c->B * c->hist_cap);
    CK(c, cudaMemcpyAsync(h.data(), c->d_hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const size_t first = c->samples.size() - n;
    for (int s = 0; s < n; ++s) {
        const auto& smp = c->samples[first + s];
        const int slot = (int)((smp.first / c->cfg.obs_every) % c->hist_cap);
        for (int b = 0; b < c->B; ++b)
            fill_obs(c, h.data() + ((size_t)slot * c->B + b) * kHistFields, smp.first, smp.second, out + (size_t)s * c->B + b);
    }
    return MD_OK;
}

md_status md_clear_history(md_ctx* c) {
    if (!c) return MD_ERR_INVALID;
    c->samples.clear();
    return MD_OK;
}

md_status md_get_state(md_ctx* c, double* pos, double* vel, int64_t* step) {
    if (!c) return MD_ERR_INVALID;
    double* st = c->h_stage;
    if (pos) {
        CK(c, cudaMemcpyAsync(st, c->d_x, sizeof(double) * 3 * c->npad, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        unpack(c, st, pos);
    }
    if (vel) {
        CK(c, cudaMemcpyAsync(st, c->d_v, sizeof(double) * 3 * c->npad, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        unpack(c, st, vel);
    }
    if (step) *step = c->step;
    return MD_OK;
}

md_status md_set_state(md_ctx* c, const double* pos, const double* vel, int64_t step) {
    if (!c || !pos || !vel) return MD_ERR_INVALID;
    if (step < 0) return fail(c, MD_ERR_INVALID, "step < 0");
    if (!finite_all(pos, 3 * c->ntot) || !finite_all(vel, 3 * c->ntot))
        return fail(c, MD_ERR_INVALID, "non-finite position or velocity");
    md_status st = upload_state(c, pos, vel);
    if (st != MD_OK) return st;
    CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream));
    c->step = step;
    st = recompute_forces(c, false);
    if (st != MD_OK) return st;
    return check_status(c);
}

md_status md_energy_forces_device(md_ctx* c, double* epot_dev, double* forces_dev) {
    if (!c) return MD_ERR_INVALID;
    md_status st = evaluate(c, true);
    if (st != MD_OK) return st;
    if (epot_dev || forces_dev)
        CK(c, launch_export_forces(c->dev, c->d_off, forces_dev, epot_dev, c->hist_cap, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_status(c);
}

md_status md_get_state_device(md_ctx* c, double* pos_dev, double* vel_dev, int64_t* step) {
    if (!c) return MD_ERR_INVALID;
    if (pos_dev || vel_dev) {
        CK(c, launch_export(c->dev, c->d_off, pos_dev, vel_dev, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    if (step) *step = c->step;
    return MD_OK;
}

md_status md_set_state_device(md_ctx* c, const double* pos_dev, const double* vel_dev, int64_t step) {
    if (!c || !pos_dev || !vel_dev) return MD_ERR_INVALID;
    if (step < 0) return fail(c, MD_ERR_INVALID, "step < 0");
    // validate first, so that a rejected state leaves the context as it was
    CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream));
    CK(c, launch_check_input(pos_dev, vel_dev, nullptr, c->ntot, c->d_status, c->stream));
    int32_t flag = 0;
    CK(c, cudaMemcpyAsync(&flag, c->d_status, sizeof flag, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (flag & invalid_input_bit()) {
        CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream));
        return fail(c, MD_ERR_INVALID, "non-finite position or velocity");
    }
    CK(c, launch_import(c->dev, c->d_off, pos_dev, vel_dev, nullptr, c->stream));
    c->step = step;
    md_status st = recompute_forces(c, false);
    if (st != MD_OK) return st;
    return check_status(c);
}

md_status md_recenter(md_ctx* c) {
    if (!c) return MD_ERR_INVALID;
    md_status st = recompute_forces(c, true);
    if (st != MD_OK) return st;
    return check_status(c);
}

md_status md_get_launch(const md_ctx* c, int32_t which, int32_t* ipt, int32_t* warps, int32_t* cluster) {
    if (!c || which < 0 || which > 1) return MD_ERR_INVALID;
    if (ipt) *ipt = c->shape[which].ipt;
    if (warps) *warps = c->shape[which].warps;
    if (cluster) *cluster = c->shape[which].cluster;
    return MD_OK;
}

md_status md_set_launch(md_ctx* c, int32_t which, int32_t ipt, int32_t warps, int32_t cluster) {
    if (!c || which < 0 || which > 1) return MD_ERR_INVALID;
    Shape s{ipt, warps, cluster};
    if (!shape_ok(s, which))
        return fail(c, MD_ERR_INVALID, "launch shape (%d,%d,%d) not supported", ipt, warps, cluster);
    c->shape[which] = s;
    drop_graphs(c);
    return MD_OK;
}

md_status md_time_passes(md_ctx* c, int32_t reps, double* ms_d, double* ms_f, double* pairs) {
    if (!c || reps < 1) return MD_ERR_INVALID;
    const Dev& d = c->dev;
    int n0, n1;
    const Item* i0 = items_for(c, c->shape[0], &n0);
    const Item* i1 = items_for(c, c->shape[1], &n1);
    const bool cells = c->path == 1, vl = c->path == 2;
    auto density = [&]() {
        return vl ? launch_v_density(d, 0, c->stream)
                  : cells ? launch_cell_density(d, 0, c->stream) : launch_density(d, i0, n0, c->shape[0], 0, c->stream);
    };
    auto force = [&]() {
        return vl ? launch_v_force(d, 0, 0, 0, c->stream)
                  : cells ? launch_cell_force(d, 0, 0, 0, c->stream)
                          : launch_force(d, i1, n1, c->shape[1], 0, 0, 0, c->stream);
    };
    CK(c, launch_mirror(d, c->stream));
    if (cells || vl) CK(c, launch_cell_build(d, c->stream));
    if (vl) CK(c, launch_v_rebuild(d, 0, 0, c->stream));
    for (int w = 0; w < 3; ++w) {
        CK(c, density());
        CK(c, force());
    }
    // reps launches back to back between one pair of events: consecutive launches overlap through
    // programmatic dependent launch exactly as they do inside the step graph, so the mean is the
    // pass's cost within a step (one event pair per launch would add a serialising gap to each)
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    double td = 0, tf = 0;
    md_status st = MD_OK;
    for (int which = 0; which < 2 && st == MD_OK; ++which) {
        cudaEventRecord(e0, c->stream);
        for (int k = 0; k < reps && st == MD_OK; ++k)
            if ((which == 0 ? density() : force()) != cudaSuccess) st = MD_ERR_CUDA;
        cudaEventRecord(e1, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) st = MD_ERR_CUDA;
        float ms = 0;
        if (st == MD_OK) cudaEventElapsedTime(&ms, e0, e1);
        (which == 0 ? td : tf) = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MD_OK) return fail(c, st, "pass launch failed while timing: %s", cudaGetErrorString(cudaGetLastError()));
    if (ms_d) *ms_d = td / reps;
    if (ms_f) *ms_f = tf / reps;
    if (pairs && vl && c->nqmax > 0) {  // quad lists: 4 pairs per listed atom, 12 within each quad
        int32_t nq = 0;
        std::vector<int32_t> cnt(c->nqmax);
        CK(c, cudaMemcpyAsync(&nq, c->d_q_n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaMemcpyAsync(cnt.data(), c->d_q_count, sizeof(int32_t) * c->nqmax, cudaMemcpyDeviceToHost,
                              c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        double p = 0;
        for (int q = 0; q < nq && q < c->nqmax; ++q) p += 4.0 * cnt[q] + 12.0;
        *pairs = p;
    } else if (pairs && vl) {  // half-list entries: each an unordered pair, i.e. two ordered pairs
        std::vector<int32_t> cnt(c->ntot);
        CK(c, cudaMemcpyAsync(cnt.data(), c->d_vcount, sizeof(int32_t) * c->ntot, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        double p = 0;
        for (int32_t n : cnt) p += 2.0 * n;
        *pairs = p;
    } else if (pairs && !cells) {
        double p = 0;
        for (int s : c->sizes) p += (double)s * (double)(s - 1);
        *pairs = p;
    } else if (pairs) {
        // pairs tested: every atom of a home octant against every atom of the 5 x 5 x 5 octants
        // around it (itself included), as binned at the current positions
        std::vector<int32_t> oct((size_t)9 * c->n_cells);
        CK(c, cudaMemcpyAsync(oct.data(), c->d_cell_oct, sizeof(int32_t) * 9 * c->n_cells, cudaMemcpyDeviceToHost,
                              c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        auto noct = [&](const CellGrid& g, int X, int Y, int Z) -> int64_t {  // octant coordinates in the grid
            if (X < 0 || Y < 0 || Z < 0 || X >= 2 * g.G || Y >= 2 * g.G || Z >= 2 * g.G) return 0;
            const int cc = g.off + ((Z / 2) * g.G + Y / 2) * g.G + X / 2, o = (X & 1) | ((Y & 1) << 1) | ((Z & 1) << 2);
            return oct[(size_t)cc * 9 + o + 1] - oct[(size_t)cc * 9 + o];
        };
        double p = 0;
        for (const CellGrid& g : c->grids)
            for (int Z = 0; Z < 2 * g.G; ++Z)
                for (int Y = 0; Y < 2 * g.G; ++Y)
                    for (int X = 0; X < 2 * g.G; ++X) {
                        const int64_t n = noct(g, X, Y, Z);
                        if (n == 0) continue;
                        int64_t nbr = 0;
                        for (int dz = -2; dz <= 2; ++dz)
                            for (int dy = -2; dy <= 2; ++dy)
                                for (int dx = -2; dx <= 2; ++dx) nbr += noct(g, X + dx, Y + dy, Z + dz);
                        p += (double)n * (double)nbr;
                    }
        *pairs = p;
    }
    return MD_OK;
}

md_status md_autotune(md_ctx* c, int32_t reps) {
    if (!c || reps < 1) return MD_ERR_INVALID;
    if (c->path >= 1 || c->half) return MD_OK;  // the cell, list and each-pair-once kernels have one launch shape
    const Dev& d = c->dev;
    // cluster sizes that are not powers of two let a small work list fill the 152 SMs more evenly
    const int ipts[3] = {1, 2, 4}, warps[4] = {2, 4, 8, 16}, clus[7] = {1, 2, 3, 4, 5, 6, 8};
    // Phase 1: every shape of each pass timed alone (CUDA events over reps launches).
    std::vector<std::pair<float, Shape>> timed[2];
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    CK(c, launch_mirror(d, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int which = 0; which < 2; ++which)
        for (int ip : ipts)
            for (int w : warps)
                for (int cl : clus) {
                    Shape s{ip, w, cl};
                    if (!shape_ok(s, which)) continue;  // e.g. four i-atoms per thread: density only, >= 4 warps
                    int n;
                    const Item* it = items_for(c, s, &n);
                    auto run = [&]() {
                        return which == 0 ? launch_density(d, it, n, s, 0, c->stream)
                                          : launch_force(d, it, n, s, 0, 0, 0, c->stream);
                    };
                    // feasibility: the cluster shape must be schedulable
                    if (run() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
                        cudaGetLastError();
                        continue;
                    }
                    run();
                    cudaEventRecord(e0, c->stream);
                    for (int k = 0; k < reps; ++k) run();
                    cudaEventRecord(e1, c->stream);
                    CK(c, cudaEventSynchronize(e1));
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    timed[which].push_back({ms, s});
                }
    for (int which = 0; which < 2; ++which) {
        if (timed[which].empty()) return fail(c, MD_ERR_CUDA, "autotune: no launch shape could run");
        std::sort(timed[which].begin(), timed[which].end(),
                  [](const std::pair<float, Shape>& a, const std::pair<float, Shape>& b) { return a.first < b.first; });
    }
    // Phase 2: the fastest shapes of each pass combined and timed where they run, inside the
    // captured MD step graph (kernels of consecutive passes overlap through programmatic
    // dependent launch, which depends on both shapes). The state is saved and restored.
    const size_t nb = sizeof(double) * 3 * c->npad;
    const size_t fb = (size_t)elem_size(c) * 3 * c->npad;
    void *sx = nullptr, *sv = nullptr, *sf = nullptr;
    CK(c, dmalloc(c, &sx, nb));
    CK(c, dmalloc(c, &sv, nb));
    CK(c, dmalloc(c, &sf, fb));
    CK(c, cudaMemcpyAsync(sx, c->d_x, nb, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(sv, c->d_v, nb, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(sf, c->d_f, fb, cudaMemcpyDeviceToDevice, c->stream));
    const int64_t step_saved = c->step;
    const double time_saved = c->time_fs;
    const int obs_saved = c->cfg.obs_every;
    const auto samples_saved = c->samples;
    c->cfg.obs_every = 0;
    const int K = 6, M = 16;
    Shape best[2] = {timed[0][0].second, timed[1][0].second};
    float best_t = 1e30f;
    md_status st = MD_OK;
    md_thermostat nve{};
    nve.kind = MD_NVE;
    // two rounds over the combinations, each keeping its best time: a combination must be slow twice to
    // lose, which keeps one noisy measurement from deciding the shapes
    for (int round = 0; round < 2 && st == MD_OK; ++round)
    for (int a = 0; a < std::min<int>(K, (int)timed[0].size()) && st == MD_OK; ++a)
        for (int b = 0; b < std::min<int>(K, (int)timed[1].size()) && st == MD_OK; ++b) {
            c->shape[0] = timed[0][a].second;
            c->shape[1] = timed[1][b].second;
            drop_graphs(c);
            st = md_step(c, M, 0.5, &nve);  // capture + warm-up
            if (st != MD_OK) break;
            cudaEventRecord(e0, c->stream);
            for (int k = 0; k < 3 && st == MD_OK; ++k) st = md_step(c, M, 0.5, &nve);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = MD_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == MD_OK && ms < best_t) {
                best_t = ms;
                best[0] = c->shape[0];
                best[1] = c->shape[1];
            }
        }
    c->cfg.obs_every = obs_saved;
    c->step = step_saved;
    c->time_fs = time_saved;
    c->samples = samples_saved;
    CK(c, cudaMemcpyAsync(c->d_x, sx, nb, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->d_v, sv, nb, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->d_f, sf, fb, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    dfree(c, sx);
    dfree(c, sv);
    dfree(c, sf);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MD_OK) return st;
    c->shape[0] = best[0];
    c->shape[1] = best[1];
    drop_graphs(c);
    cache_store(c->cfg.tune_cache, tune_key(c), c->shape);
    // forces, densities and mirror of the restored state under the chosen shapes
    st = evaluate(c, false);
    if (st != MD_OK) return st;
    CK(c, cudaStreamSynchronize(c->stream));
    return MD_OK;
}

md_status md_get_path(const md_ctx* c, int32_t* path) {
    if (!c || !path) return MD_ERR_INVALID;
    *path = c->path == 2 ? MD_PATH_VERLET
                         : (c->path == 1 ? MD_PATH_CELLS : (c->half ? MD_PATH_ALLPAIRS_HALF : MD_PATH_ALLPAIRS));
    return MD_OK;
}

md_status md_launch_counts(const md_ctx* c, int32_t* per_step, int32_t* per_chunk) {
    if (!c) return MD_ERR_INVALID;
    // lists: positions, cell build (FP64 3: clear, bin, sort; MIXED 1: bin, in a step), list build (MIXED scan,
    // order, list; FP64 build, sort, reverse sort, commit), passes (MIXED 2; FP64 compaction, 2 passes, 2 gathers)
    // (MIXED: the position kernel runs once per chunk, and every step with Berendsen)
    if (per_step) *per_step = c->path == 2 ? (c->nqmax > 0 ? 6 : 13) : (c->path == 1 ? 5 : (c->half ? 4 : 2));
    if (per_chunk) *per_chunk = c->path == 2 && c->nqmax > 0 ? 4 : 3;
    return MD_OK;
}

md_status md_philox4x32_10(const uint32_t* in, uint32_t* out, int32_t count) {
    if (count < 0 || (count > 0 && (!in || !out))) return fail(nullptr, MD_ERR_INVALID, "bad arguments");
    if (count == 0) return MD_OK;
    uint32_t *din = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&din, sizeof(uint32_t) * 6 * count);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint32_t) * 4 * count);
    if (e == cudaSuccess) e = cudaMemcpy(din, in, sizeof(uint32_t) * 6 * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(din, dout, count, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint32_t) * 4 * count, cudaMemcpyDeviceToHost);
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, MD_ERR_CUDA, "philox: %s", cudaGetErrorString(e));
    return MD_OK;
}

md_status md_langevin_normals(uint64_t seed, uint32_t cluster, int64_t step, int32_t n_atoms, int32_t precision,
                              double* out) {
    if (n_atoms < 0 || (n_atoms > 0 && !out)) return fail(nullptr, MD_ERR_INVALID, "bad arguments");
    if (n_atoms == 0) return MD_OK;
    double* dout = nullptr;
    cudaError_t e = cudaMalloc(&dout, sizeof(double) * 3 * n_atoms);
    if (e == cudaSuccess) e = launch_normals(seed, cluster, step, n_atoms, precision, dout, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToHost);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, MD_ERR_CUDA, "normals: %s", cudaGetErrorString(e));
    return MD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- structural observables (Sec. III)
namespace {
constexpr int kMaxBins = 8192;  // histogram bins (shared-memory counters of one CTA)

md_status struct_alloc(md_ctx* c) {
    if (c->sb.com) return MD_OK;
    const size_t np = (size_t)c->npad, B = (size_t)c->B;
    StructBufs& b = c->sb;
    CK(c, dmalloc(c, &b.com, sizeof(double) * 3 * B));
    CK(c, dmalloc(c, &b.core, sizeof(int32_t) * np));
    CK(c, dmalloc(c, &b.ncore, sizeof(int32_t) * B));
    CK(c, dmalloc(c, &b.ref, sizeof(double) * 3 * np));
    CK(c, dmalloc(c, &b.ref_com, sizeof(double) * 3 * B));
    CK(c, dmalloc(c, &b.sel, np));
    CK(c, dmalloc(c, &b.msd, sizeof(double) * B));
    CK(c, dmalloc(c, &b.nsel, sizeof(int32_t) * B));
    CK(c, dmalloc(c, &b.nb, sizeof(int32_t) * kNbCap * np));
    CK(c, dmalloc(c, &b.nnb, sizeof(int32_t) * np));
    CK(c, dmalloc(c, &b.cls, np));
    CK(c, dmalloc(c, &b.counts, sizeof(int32_t) * 4 * B));
    CK(c, dmalloc(c, &b.capped, sizeof(int32_t) * B));
    CK(c, cudaMemsetAsync(b.nnb, 0, sizeof(int32_t) * np, c->stream));
    CK(c, cudaMemsetAsync(b.cls, 0, np, c->stream));
    return MD_OK;
}
}  // namespace

extern "C" {

md_status md_rdf(md_ctx* c, double r_core_A, double bin_A, int32_t nbins, int64_t* counts, int32_t* n_core) {
    if (!c || !counts) return MD_ERR_INVALID;
    if (!(std::isfinite(r_core_A) && r_core_A >= 0) || !(std::isfinite(bin_A) && bin_A > 0))
        return fail(c, MD_ERR_INVALID, "r_core_A must be >= 0 and bin_A > 0");
    if (nbins < 1 || nbins > kMaxBins) return fail(c, MD_ERR_INVALID, "nbins must be in 1..%d", kMaxBins);
    md_status st = struct_alloc(c);
    if (st != MD_OK) return st;
    if (nbins > c->sb_nbins) {
        dfree(c, c->sb.hist);
        c->sb.hist = nullptr;
        c->sb_nbins = 0;
        CK(c, dmalloc(c, &c->sb.hist, sizeof(unsigned long long) * (size_t)c->B * nbins));
        c->sb_nbins = nbins;
    }
    CK(c, cudaMemsetAsync(c->sb.hist, 0, sizeof(unsigned long long) * (size_t)c->B * nbins, c->stream));
    int maxn = 1;
    for (int s : c->sizes) maxn = std::max(maxn, s);
    const int Y = std::max(1, std::min(128, (maxn + 511) / 512));
    CK(c, launch_rdf(c->dev, c->sb, r_core_A, bin_A, nbins, Y, c->stream));
    CK(c, cudaMemcpyAsync(counts, c->sb.hist, sizeof(int64_t) * (size_t)c->B * nbins, cudaMemcpyDeviceToHost,
                          c->stream));
    if (n_core)
        CK(c, cudaMemcpyAsync(n_core, c->sb.ncore, sizeof(int32_t) * c->B, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return MD_OK;
}

md_status md_msd_reference(md_ctx* c, double r_core_A) {
    if (!c) return MD_ERR_INVALID;
    if (!std::isfinite(r_core_A)) return fail(c, MD_ERR_INVALID, "r_core_A must be finite");
    md_status st = struct_alloc(c);
    if (st != MD_OK) return st;
    CK(c, launch_msd_ref(c->dev, c->sb, r_core_A, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->msd_ref = true;
    return MD_OK;
}

md_status md_msd(md_ctx* c, double* msd_A2, int32_t* n_atoms) {
    if (!c || !msd_A2) return MD_ERR_INVALID;
    if (!c->msd_ref) return fail(c, MD_ERR_STATE, "no reference configuration: call md_msd_reference first");
    CK(c, launch_msd(c->dev, c->sb, c->stream));
    CK(c, cudaMemcpyAsync(msd_A2, c->sb.msd, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->stream));
    if (n_atoms)
        CK(c, cudaMemcpyAsync(n_atoms, c->sb.nsel, sizeof(int32_t) * c->B, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return MD_OK;
}

md_status md_cna(md_ctx* c, double r_nb_A, int32_t* counts, int8_t* cls, int32_t* capped) {
    if (!c || !counts) return MD_ERR_INVALID;
    if (!(std::isfinite(r_nb_A) && r_nb_A > 0)) return fail(c, MD_ERR_INVALID, "r_nb_A must be > 0");
    md_status st = struct_alloc(c);
    if (st != MD_OK) return st;
    CK(c, cudaMemsetAsync(c->sb.counts, 0, sizeof(int32_t) * 4 * c->B, c->stream));
    CK(c, cudaMemsetAsync(c->sb.capped, 0, sizeof(int32_t) * c->B, c->stream));
    CK(c, launch_cna(c->dev, c->sb, r_nb_A, c->stream));
    CK(c, cudaMemcpyAsync(counts, c->sb.counts, sizeof(int32_t) * 4 * c->B, cudaMemcpyDeviceToHost, c->stream));
    if (capped)
        CK(c, cudaMemcpyAsync(capped, c->sb.capped, sizeof(int32_t) * c->B, cudaMemcpyDeviceToHost, c->stream));
    int8_t* st8 = reinterpret_cast<int8_t*>(c->h_stage);
    if (cls) CK(c, cudaMemcpyAsync(st8, c->sb.cls, (size_t)c->npad, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (cls)
        for (int b = 0; b < c->B; ++b)
            for (int a = 0; a < c->sizes[b]; ++a) cls[c->off[b] + a] = st8[c->poff[b] + a];
    return MD_OK;
}

}  // extern "C"
