// api.cu -- host side of libiblb: the C ABI declared in include/iblb.h.
//
// A context owns pooled device buffers for all of its droplets, a CUDA
// stream of its own, and (by default) two captured CUDA graphs of one time
// step (one per population buffer parity).  The step enqueues, in order:
//   (a1) nodal forces + binning, (a2) bin scan, fill, deterministic gather-
//   spread, (a3) in/out ray casting when some droplet has lambda != 1,
//   (a4) fused stream-collide, (a5) interpolation + advection, (a6) FP64 mesh
//   reductions + volume correction when requested.
#include <math.h>
#include <stdio.h>

#include <cmath>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/iblb.h"
#include "iblb_internal.h"

using namespace iblb;

namespace {

const char *kVersion = "iblb 0.1 (sm_103a)";
thread_local std::string g_create_error;

const double kWh[Q] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

size_t storage_bytes(int storage) { return storage == IBLB_STORE_F32 ? 4 : 2; }

struct Membrane {
    std::vector<double> xyz;   // positions as stored on the device (host copy, refreshed on rebuild)
    double corr[NRED] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // its row of red_out (pending correction)
    std::vector<double> ref;   // the elastic reference: the mesh as given to iblb_set_membrane
    std::vector<int> tri;      // local node indices
    bool set = false;
    double V0 = 0.0;
};

}  // namespace

struct iblb_ctx {
    int ndrops = 0;
    int storage = 0;
    std::vector<iblb_lattice_desc> lat;
    std::vector<iblb_physics_desc> phys;
    std::vector<Drop> drops;
    std::vector<Membrane> mem;
    bool mem_dirty = false;
    bool any_vartau = false, any_volcorr = false;
    Arrays A{};
    Drop *d_drops = nullptr;
    void *fbuf[2] = {nullptr, nullptr};
    int cur = 0;
    int *d_tri = nullptr, *d_adj_start = nullptr, *d_adj = nullptr;
    int4 *d_ring = nullptr, *d_ring8 = nullptr;
    float4 *d_fref = nullptr;
    int n_red_chunks = 0, mass_blocks = 0;
    double *d_mass = nullptr;
    cudaStream_t user = nullptr, stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaStream_t side = nullptr;   // stream-collide of the groups far from the band
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool split_lb = false;         // run those groups concurrently with the membrane kernels
    int lb_far_blocks_per_sm = 1;
    cudaEvent_t ph[IBLB_NPHASE + 1] = {};
    bool graphs = false;           // eager launches chained by programmatic dependent launch are
                                   // faster on GB300 than graph replay (81 against 84 us at 128^3)
    bool fused_ib = false;         // membrane work as two cooperative kernels
    bool pdl = true;               // programmatic dependent launch between the kernels of a step
    int profile = 0;               // 0 off, 1 every phase, 2 whole step only
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool gvalid[2] = {false, false};
    int graph_chunk = 1;           // steps per replayed graph (K-step graphs when > 1)
    cudaGraphExec_t gchunk[2] = {nullptr, nullptr};   // K steps from buffer parity 0 / 1
    double ph_ms[IBLB_NPHASE] = {};
    double step_ms = 0.0;
    int64_t prof_steps = 0;
    int64_t step_count = 0;
    LaunchCfg cfg{0, 2, 148, 3, 1, 768};
    int *h_status = nullptr;     // pinned, 4 per droplet
    double *obs_scr = nullptr;   // scratch of the mesh observation kernels
    int64_t obs_scr_n = 0;
    unsigned long long *d_trace = nullptr;   // per-warp stamps of iblb_trace_step (allocated by its first call)
    double *d_stage = nullptr;   // x, y, z per node of one droplet: node uploads and downloads
    int64_t d_stage_n = 0;
    double *h_obs = nullptr;     // pinned: 32 raw observation doubles, then one mass per droplet
    cudaEvent_t ev_copy = nullptr;   // a node upload has left the caller's buffer
    std::string err;
};

namespace {

// NVTX range around a public call, for timeline tools (no cost without one)
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
};

int fail(iblb_ctx *c, int code, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_create_error = msg;
    return code;
}

// A failed CUDA call is reported and its error cleared from the runtime's
// last-error slot, so that it does not surface again in a later, unrelated
// call (of this or another context).  Sticky errors stay sticky.
#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            (void)cudaGetLastError();                                                             \
            return fail(c, IBLB_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
        }                                                                                         \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0)
        n = 1;
    return cudaMalloc((void **)p, n * sizeof(T));
}

void dfree(void *p)
{
    if (p)
        cudaFree(p);
}

// order the context's stream after the caller's, and the caller's after ours
void enter(iblb_ctx *c)
{
    cudaEventRecord(c->ev_in, c->user);
    cudaStreamWaitEvent(c->stream, c->ev_in, 0);
}
void leave(iblb_ctx *c)
{
    cudaEventRecord(c->ev_out, c->stream);
    cudaStreamWaitEvent(c->user, c->ev_out, 0);
}

// enter() on construction, leave() on every way out of the scope, early
// error returns included, so that the caller's stream is always ordered
// after whatever the call managed to queue
struct Entered {
    iblb_ctx *c;
    explicit Entered(iblb_ctx *ctx) : c(ctx) { enter(c); }
    ~Entered() { leave(c); }
    Entered(const Entered &) = delete;
    Entered &operator=(const Entered &) = delete;
};

void invalidate_graphs(iblb_ctx *c)
{
    for (int p = 0; p < 2; ++p) {
        if (c->gexec[p])
            cudaGraphExecDestroy(c->gexec[p]);
        c->gexec[p] = nullptr;
        c->gvalid[p] = false;
        if (c->gchunk[p])
            cudaGraphExecDestroy(c->gchunk[p]);
        c->gchunk[p] = nullptr;
    }
}

int check_desc(const iblb_lattice_desc &l, const iblb_physics_desc &p, std::string &why)
{
    if (l.nx < 8 || l.ny < 8 || l.nz < 8) {
        why = "box sides must be >= 8";
        return 0;
    }
    if (l.nx > 8188 || l.ny > 8188 || l.nz > 4094) {
        why = "box sides must be at most 8188 (x, y) and 4094 (z) cells";
        return 0;
    }
    if ((int64_t)l.nx * l.ny * l.nz > ((int64_t)1 << 31) / 2) {
        why = "box too large (cells must stay below 2^30)";
        return 0;
    }
    if (!(l.tau_out > 0.5)) {
        why = "tau_out must exceed 1/2";
        return 0;
    }
    if (!(l.lambda > 0.0)) {
        why = "lambda must be positive";
        return 0;
    }
    if (!(l.rho0 > 0.0)) {
        why = "rho0 must be positive";
        return 0;
    }
    if (l.storage < 0 || l.storage > 2) {
        why = "unknown storage";
        return 0;
    }
    if (l.walls != 0 && l.walls != 1) {
        why = "walls must be 0 or 1";
        return 0;
    }
    if (p.sigma < 0.0) {
        why = "sigma must be >= 0";
        return 0;
    }
    if (p.wetting < 0 || p.wetting > 2) {
        why = "unknown wetting model";
        return 0;
    }
    if (p.wetting) {
        if (!(p.xi > 0.0) || p.n <= p.m || p.m < 1 || p.n > 32) {
            why = "wetting needs xi > 0 and 32 >= n > m >= 1";
            return 0;
        }
        if (!l.walls) {
            why = "wetting needs walls";
            return 0;
        }
        if (p.h_min_frac < 0.0) {
            why = "h_min_frac must be >= 0";
            return 0;
        }
    }
    if (!(p.shear_modulus >= 0.0) || !(p.area_modulus >= 0.0)) {
        why = "the membrane moduli must be >= 0";
        return 0;
    }
    return 1;
}

// Closed, orientable, Euler characteristic 2 and positive volume.
int validate_mesh(const double *xyz, int n, const int32_t *tri, int nt, std::string &why, double *V)
{
    if (n < 4 || nt < 4) {
        why = "a closed mesh needs at least 4 nodes and 4 faces";
        return 0;
    }
    std::map<std::pair<int, int>, int> directed;
    std::vector<int> used(n, 0);
    for (int t = 0; t < nt; ++t) {
        const int a = tri[3 * t], b = tri[3 * t + 1], cc = tri[3 * t + 2];
        if (a < 0 || b < 0 || cc < 0 || a >= n || b >= n || cc >= n) {
            why = "face index out of range";
            return 0;
        }
        if (a == b || b == cc || a == cc) {
            why = "degenerate face";
            return 0;
        }
        const int v[3] = {a, b, cc};
        for (int k = 0; k < 3; ++k) {
            used[v[k]] = 1;
            if (++directed[{v[k], v[(k + 1) % 3]}] > 1) {
                why = "edge used twice in the same direction (non-manifold or inconsistent orientation)";
                return 0;
            }
        }
    }
    for (auto &kv : directed)
        if (!directed.count({kv.first.second, kv.first.first})) {
            why = "open mesh: an edge has one face only";
            return 0;
        }
    for (int j = 0; j < n; ++j)
        if (!used[j]) {
            why = "node not used by any face";
            return 0;
        }
    const int64_t E = (int64_t)directed.size() / 2;
    if ((int64_t)n - E + nt != 2) {
        why = "Euler characteristic is not 2";
        return 0;
    }
    for (int k = 0; k < 3 * n; ++k)
        if (!std::isfinite(xyz[k])) {
            why = "non-finite node position";
            return 0;
        }
    double vol = 0.0;
    for (int t = 0; t < nt; ++t) {
        const double *a = xyz + 3 * tri[3 * t], *b = xyz + 3 * tri[3 * t + 1], *cc = xyz + 3 * tri[3 * t + 2];
        vol += a[0] * (b[1] * cc[2] - b[2] * cc[1]) + a[1] * (b[2] * cc[0] - b[0] * cc[2]) +
               a[2] * (b[0] * cc[1] - b[1] * cc[0]);
    }
    vol /= 6.0;
    if (!(vol > 0.0)) {
        why = "mesh volume not positive (faces must be counter-clockwise seen from outside)";
        return 0;
    }
    *V = vol;
    return 1;
}

void fill_drop_params(Drop &D, const iblb_lattice_desc &l, const iblb_physics_desc &p)
{
    D.nx = l.nx;
    D.ny = l.ny;
    D.nz = l.nz;
    D.walls = l.walls;
    D.nzf = l.walls ? l.nz - 2 : l.nz;
    D.tx = (l.nx + 3) / 4;
    D.ty = (l.ny + 3) / 4;
    D.tz = (D.nzf + 3) / 4;
    D.ntiles = D.tx * D.ty * D.tz;
    D.cells = (int64_t)l.nx * l.ny * D.nzf;
    const double tin = 0.5 + l.lambda * (l.tau_out - 0.5);
    D.tau_out = (float)l.tau_out;
    D.tau_in = (float)tin;
    D.omega_out = (float)(1.0 / l.tau_out);
    D.omega_in = (float)(1.0 / tin);
    D.vartau = l.lambda != 1.0;
    D.rho0 = (float)l.rho0;
    for (int k = 0; k < 3; ++k)
        D.bf[k] = (float)l.body_force[k];
    D.sigma = (float)p.sigma;
    D.wetting = p.wetting != IBLB_WET_OFF;
    double A = 0.0;
    if (p.wetting == IBLB_WET_THETA)
        A = p.sigma * (double)((p.m - 1) * (p.n - 1)) / ((double)(p.n - p.m) * p.xi) *
            (1.0 + cos(p.theta_eq_deg * M_PI / 180.0));
    else if (p.wetting == IBLB_WET_RAW)
        A = p.A;
    D.A = (float)A;
    D.xi = (float)(p.xi > 0 ? p.xi : 1.0);
    D.hmin = (float)(p.h_min_frac * (p.xi > 0 ? p.xi : 1.0));
    D.n = p.n;
    D.m = p.m;
    D.volcorr = p.volume_correction != 0;
    D.ks = (float)p.shear_modulus;
    D.ka = (float)p.area_modulus;
}

// shared memory a block of the stream-collide kernel may give its stages: the
// opt-in maximum of sm_100 and later (227 KB) less 1 KB for its static part
constexpr int64_t kLbSmemOptin = 227 * 1024 - 1024;

// as many of the asked pipeline stages as fit the block's shared memory
void fit_stages(iblb_ctx *c)
{
    while (c->cfg.lb_stages > 2 && (int64_t)c->cfg.lb_stages * c->A.lb_stage_bytes > kLbSmemOptin)
        --c->cfg.lb_stages;
}

// Offsets of cells, tiles, columns, launch blocks for the current launch shape.
void layout(iblb_ctx *c)
{
    int64_t cell0 = 0, tile0 = 0, col0 = 0, pcell0 = 0, row0 = 0, trow0 = 0;
    int lb0 = 0, mb0 = 0, stage = 0;
    const int sb = (int)storage_bytes(c->storage);
    for (auto &D : c->drops) {
        D.cell0 = cell0;
        D.tile0 = tile0;
        D.trow0 = trow0;
        D.col0 = col0;
        // rows padded to 16 bytes of population storage (and of the float
        // force / velocity rows, whose pitch is the same)
        const int align = 16 / sb;
        D.pitch = (D.nx + align - 1) / align * align;
        D.pcells = (int64_t)D.pitch * D.ny * D.nzf;
        D.pcell0 = pcell0;
        D.row0 = row0;
        D.lb_rows = std::min(D.ny, c->cfg.lb_group_cells > 0
                                       ? std::max(1, (c->cfg.lb_group_cells + D.nx / 2) / D.nx)
                                       : c->cfg.lb_row_mult * lb_rows_per_group(D.nx));
        // two stages of the group must fit the opt-in shared memory of a block
        while (D.lb_rows > 1 && 2 * (int64_t)lb_stage_bytes(D.lb_rows, D.pitch, sb) > kLbSmemOptin)
            --D.lb_rows;
        D.lb_gpp = (D.ny + D.lb_rows - 1) / D.lb_rows;
        D.lb_block0 = lb0;
        D.lb_nblocks = D.lb_gpp * D.nzf;
        D.mass_block0 = mb0;
        D.mass_nblocks = (int)((D.cells + MASS_CELLS_PER_BLOCK - 1) / MASS_CELLS_PER_BLOCK);
        stage = std::max(stage, lb_stage_bytes(D.lb_rows, D.pitch, sb));
        cell0 += D.cells;
        pcell0 += D.pcells;
        row0 += (int64_t)D.ny * D.nzf;
        tile0 += D.ntiles;
        trow0 += (int64_t)D.ty * D.tz;
        col0 += (int64_t)D.nx * D.ny;
        lb0 += D.lb_nblocks;
        mb0 += D.mass_nblocks;
    }
    c->A.total_cells = cell0;
    c->A.total_pcells = pcell0;
    c->A.total_rows = row0;
    c->A.total_tiles = tile0;
    c->A.total_trows = trow0;
    c->A.total_cols = col0;
    c->A.lb_blocks_total = lb0;
    c->A.lb_stage_bytes = stage;
    c->mass_blocks = mb0;
    fit_stages(c);
}

int upload_drops(iblb_ctx *c)
{
    CK(cudaMemcpyAsync(c->d_drops, c->drops.data(), sizeof(Drop) * c->ndrops, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IBLB_OK;
}

// Pull the current device node positions into the host copies.
int download_nodes(iblb_ctx *c)
{
    if (!c->A.total_nodes)
        return IBLB_OK;
    const int N = c->A.total_nodes;
    std::vector<double> x(N), y(N), z(N);
    CK(cudaMemcpyAsync(x.data(), c->A.qx, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(y.data(), c->A.qy, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(z.data(), c->A.qz, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    std::vector<double> ro((size_t)NRED * c->ndrops);
    CK(cudaMemcpyAsync(ro.data(), c->A.red_out, sizeof(double) * ro.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int d = 0; d < c->ndrops; ++d) {
        const Drop &D = c->drops[d];
        if (D.nnodes)
            memcpy(c->mem[d].corr, &ro[(size_t)NRED * d], sizeof(double) * NRED);
        for (int j = 0; j < D.nnodes; ++j) {
            c->mem[d].xyz[3 * j] = x[D.node0 + j];
            c->mem[d].xyz[3 * j + 1] = y[D.node0 + j];
            c->mem[d].xyz[3 * j + 2] = z[D.node0 + j];
        }
    }
    return IBLB_OK;
}

// Node positions as FP32 pairs: hi = q rounded to FP32, lo = q - hi (exact
// in FP64) rounded to FP32; the advection writes the same split on the
// device.
void split_positions(const double *x, const double *y, const double *z, int64_t n, float4 *hi, float4 *lo)
{
    for (int64_t j = 0; j < n; ++j) {
        const float hx = (float)x[j], hy = (float)y[j], hz = (float)z[j];
        hi[j] = make_float4(hx, hy, hz, 0.0f);
        lo[j] = make_float4((float)(x[j] - (double)hx), (float)(y[j] - (double)hy), (float)(z[j] - (double)hz), 0.0f);
    }
}

void free_membrane_arrays(iblb_ctx *c)
{
    dfree(c->A.qx);
    dfree(c->A.qy);
    dfree(c->A.qz);
    dfree(c->A.px);
    dfree(c->A.py);
    dfree(c->A.pz);
    c->A.px = c->A.py = c->A.pz = nullptr;
    dfree(c->A.qh);
    dfree(c->A.ql);
    c->A.qh = c->A.ql = nullptr;
    dfree(c->A.node_drop);
    dfree(c->d_tri);
    dfree(c->A.face_drop);
    dfree(c->d_adj_start);
    dfree(c->d_adj);
    dfree(c->d_ring);
    dfree(c->d_ring8);
    c->d_ring = c->d_ring8 = nullptr;
    c->A.ring = c->A.ring8 = nullptr;
    dfree(c->d_fref);
    c->d_fref = nullptr;
    c->A.fref = nullptr;
    dfree(c->A.rec);
    dfree(c->A.clamped);
    dfree(c->A.red_part);
    dfree(c->A.red_out);
    dfree(c->A.vc_done);
    c->A.vc_done = nullptr;
    c->A.qx = c->A.qy = c->A.qz = nullptr;
    c->A.node_drop = c->A.face_drop = nullptr;
    c->d_tri = c->d_adj_start = c->d_adj = nullptr;
    c->A.tri = c->A.adj_start = c->A.adj = nullptr;
    c->A.rec = nullptr;
    c->A.clamped = nullptr;
    c->A.red_part = c->A.red_out = nullptr;
}

// (Re)build the pooled node / face / adjacency arrays from the host copies.
int rebuild_membranes(iblb_ctx *c)
{
    if (!c->mem_dirty)
        return IBLB_OK;
    free_membrane_arrays(c);
    int N = 0, NT = 0, chunks = 0;
    for (int d = 0; d < c->ndrops; ++d) {
        Drop &D = c->drops[d];
        const Membrane &M = c->mem[d];
        D.node0 = N;
        D.tri0 = NT;
        D.nnodes = M.set ? (int)(M.xyz.size() / 3) : 0;
        D.ntri = M.set ? (int)(M.tri.size() / 3) : 0;
        D.red_chunk0 = chunks;
        int nc = 0;
        if (D.nnodes) {
            nc = std::max((D.ntri + VC_ITEMS - 1) / VC_ITEMS, (D.nnodes + VC_ITEMS - 1) / VC_ITEMS);
            nc = std::max(nc, 1);
        }
        D.red_nchunks = nc;
        D.V0 = M.V0;
        D.R0 = cbrt(3.0 * M.V0 / (4.0 * M_PI));
        D.inv_n = D.nnodes ? 1.0 / D.nnodes : 0.0;
        D.inv6V0 = M.V0 > 0.0 ? 1.0 / (6.0 * M.V0) : 0.0;
        N += D.nnodes;
        NT += D.ntri;
        chunks += nc;
    }
    c->A.total_nodes = N;
    c->A.total_tri = NT;
    c->n_red_chunks = chunks;
    std::vector<double> x(N), y(N), z(N);
    std::vector<int> nd(N), tri(3 * (size_t)NT), fd(NT), start(N + 1, 0), adj;
    for (int d = 0; d < c->ndrops; ++d) {
        const Drop &D = c->drops[d];
        const Membrane &M = c->mem[d];
        for (int j = 0; j < D.nnodes; ++j) {
            x[D.node0 + j] = M.xyz[3 * j];
            y[D.node0 + j] = M.xyz[3 * j + 1];
            z[D.node0 + j] = M.xyz[3 * j + 2];
            nd[D.node0 + j] = d;
        }
        for (int t = 0; t < D.ntri; ++t) {
            for (int k = 0; k < 3; ++k) {
                tri[3 * (size_t)(D.tri0 + t) + k] = D.node0 + M.tri[3 * t + k];
                start[D.node0 + M.tri[3 * t + k] + 1]++;
            }
            fd[D.tri0 + t] = d;
        }
    }
    for (int j = 0; j < N; ++j)
        start[j + 1] += start[j];
    adj.resize(start[N] > 0 ? start[N] : 1);
    std::vector<int4> ring(adj.size()), ring8((size_t)RING8 * std::max(N, 1), make_int4(-1, -1, 0, 0));
    {
        std::vector<int> pos(start.begin(), start.end() - 1);
        for (int t = 0; t < NT; ++t)       // faces in increasing order per node
            for (int k = 0; k < 3; ++k) {
                const int e = pos[tri[3 * (size_t)t + k]]++;
                adj[e] = (t << 2) | k;
                // the other corners in counter-clockwise order after this one
                ring[e] = make_int4(tri[3 * (size_t)t + (k + 1) % 3], tri[3 * (size_t)t + (k + 2) % 3], (t << 2) | k, 0);
            }
        for (int j = 0; j < N; ++j) {
            const int v = start[j + 1] - start[j];
            for (int q = 0; q < RING8; ++q) {
                int4 en = q < v ? ring[start[j] + q] : make_int4(-1, -1, 0, 0);
                en.w = v;
                ring8[(size_t)RING8 * j + q] = en;
            }
        }
    }
    if (NT >= (1 << 29))
        return fail(c, IBLB_E_ARG, "too many faces");
    CK(dalloc(&c->A.qx, N));
    CK(dalloc(&c->A.qy, N));
    CK(dalloc(&c->A.qz, N));
    CK(dalloc(&c->A.px, N));
    CK(dalloc(&c->A.py, N));
    CK(dalloc(&c->A.pz, N));
    CK(dalloc(&c->A.qh, N));
    CK(dalloc(&c->A.ql, N));
    CK(dalloc(&c->A.node_drop, N));
    CK(dalloc(&c->d_tri, 3 * (size_t)NT));
    CK(dalloc(&c->A.face_drop, NT));
    // reference geometry of every face of an elastic droplet: S = H^-1 of the
    // Gram matrix H = [E_i . E_j] of its reference edges E1 = X1 - X0,
    // E2 = X2 - X0, and its reference area A0 = sqrt(det H) / 2
    bool elastic = false;
    for (int d = 0; d < c->ndrops; ++d)
        elastic |= c->drops[d].ks != 0.0f || c->drops[d].ka != 0.0f;
    std::vector<float4> fref;
    if (elastic) {
        fref.assign(NT > 0 ? NT : 1, make_float4(0.f, 0.f, 0.f, 1.f));
        for (int d = 0; d < c->ndrops; ++d) {
            const Drop &D = c->drops[d];
            const Membrane &M = c->mem[d];
            for (int t = 0; t < D.ntri; ++t) {
                const int *v = &M.tri[3 * (size_t)t];
                double E1[3], E2[3];
                for (int a = 0; a < 3; ++a) {
                    E1[a] = M.ref[3 * (size_t)v[1] + a] - M.ref[3 * (size_t)v[0] + a];
                    E2[a] = M.ref[3 * (size_t)v[2] + a] - M.ref[3 * (size_t)v[0] + a];
                }
                const double h11 = E1[0] * E1[0] + E1[1] * E1[1] + E1[2] * E1[2];
                const double h12 = E1[0] * E2[0] + E1[1] * E2[1] + E1[2] * E2[2];
                const double h22 = E2[0] * E2[0] + E2[1] * E2[1] + E2[2] * E2[2];
                const double det = h11 * h22 - h12 * h12;
                fref[D.tri0 + t] = make_float4((float)(h22 / det), (float)(-h12 / det), (float)(h11 / det),
                                               (float)(0.5 * sqrt(det)));
            }
        }
        CK(dalloc(&c->d_fref, fref.size()));
    }
    CK(dalloc(&c->d_adj_start, N + 1));
    CK(dalloc(&c->d_adj, adj.size()));
    CK(dalloc(&c->d_ring, ring.size()));
    CK(dalloc(&c->d_ring8, ring8.size()));
    CK(dalloc(&c->A.rec, N));
    CK(dalloc(&c->A.clamped, N));
    CK(cudaMemsetAsync(c->A.clamped, 0, N, c->stream));
    CK(dalloc(&c->A.red_part, (size_t)NRED * std::max(chunks, 1)));
    CK(dalloc(&c->A.red_out, (size_t)NRED * c->ndrops));
    CK(dalloc(&c->A.vc_done, (size_t)c->ndrops));
    CK(cudaMemsetAsync(c->A.vc_done, 0, sizeof(int) * c->ndrops, c->stream));
    c->A.tri = c->d_tri;
    c->A.adj_start = c->d_adj_start;
    c->A.adj = c->d_adj;
    c->A.ring = c->d_ring;
    c->A.ring8 = c->d_ring8;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream) : cudaSuccess;
    };
    CK(up(c->A.qx, x.data(), sizeof(double) * N));
    CK(up(c->A.qy, y.data(), sizeof(double) * N));
    CK(up(c->A.qz, z.data(), sizeof(double) * N));
    std::vector<float4> qh(N), ql(N);
    split_positions(x.data(), y.data(), z.data(), N, qh.data(), ql.data());
    CK(up(c->A.qh, qh.data(), sizeof(float4) * N));
    CK(up(c->A.ql, ql.data(), sizeof(float4) * N));
    CK(up(c->A.node_drop, nd.data(), sizeof(int) * N));
    CK(up(c->d_tri, tri.data(), sizeof(int) * tri.size()));
    CK(up(c->A.face_drop, fd.data(), sizeof(int) * NT));
    CK(up(c->d_adj_start, start.data(), sizeof(int) * (N + 1)));
    CK(up(c->d_adj, adj.data(), sizeof(int) * adj.size()));
    CK(up(c->d_ring, ring.data(), sizeof(int4) * ring.size()));
    CK(up(c->d_ring8, ring8.data(), sizeof(int4) * ring8.size()));
    if (elastic)
        CK(up(c->d_fref, fref.data(), sizeof(float4) * fref.size()));
    {   // each droplet's pending volume correction (none for a new membrane)
        std::vector<double> ro((size_t)NRED * c->ndrops);
        for (int d = 0; d < c->ndrops; ++d)
            memcpy(&ro[(size_t)NRED * d], c->mem[d].corr, sizeof(double) * NRED);
        CK(up(c->A.red_out, ro.data(), sizeof(double) * ro.size()));
    }
    c->A.fref = c->d_fref;
    CK(cudaMemsetAsync(c->A.bin_cnt, 0, sizeof(int) * c->A.total_tiles, c->stream));
    CK(cudaMemsetAsync(c->A.split_ok, 0, sizeof(int), c->stream));   // no previous band for these nodes
    c->mem_dirty = false;
    int r = upload_drops(c);
    invalidate_graphs(c);
    return r;
}

int ensure_ready(iblb_ctx *c)
{
    return rebuild_membranes(c);
}

// One time step on c->stream with population buffers (src = fbuf[par]).
int enqueue_step(iblb_ctx *c, int par, bool forces_only)
{
    cudaStream_t s = c->stream;
    c->A.pdl = c->pdl && !c->fused_ib;
    const Arrays &a = c->A;
    const bool nodes = a.total_nodes > 0;
    const bool prof = c->profile;
    // phase boundaries; "external" so that, under stream capture, they become
    // event-record nodes of the graph that the host can time after a replay
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (prof)
        CK(cudaStreamIsCapturing(s, &cap));
    auto mark = [&](int k) {
        const bool on = c->profile == 1 || (c->profile == 2 && (k == 0 || k == IBLB_NPHASE)) ||
                        (c->profile == 3 && (k == IBLB_PH_LB || k == IBLB_PH_LB + 1));
        if (!prof || !on)
            return cudaSuccess;
        return cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(c->ph[k], s, cudaEventRecordExternal)
                                                    : cudaEventRecord(c->ph[k], s);
    };
    CK(mark(0));
    // groups far from the band: on the side stream, concurrently with the
    // membrane kernels (the in/out test goes first: the far groups inside a
    // droplet need it, and the node positions are final)
    const bool split = nodes && c->split_lb && !forces_only;
    if (split) {
        CK(launch_classify(a, s));
        if (c->any_vartau) {
            CK(launch_corrected_positions(a, s));     // the force kernel has not written them yet
            CK(launch_inout(a, s));
        }
        CK(cudaEventRecord(c->ev_fork, s));
        CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        CK(launch_lb(a, c->storage, c->fbuf[par], c->fbuf[par ^ 1], c->any_vartau, c->cfg, c->side,
                     a.grp_list + a.total_rows, a.grp_cnt + 1, true, c->lb_far_blocks_per_sm));
        CK(cudaEventRecord(c->ev_join, c->side));
    }
    if (nodes && c->fused_ib) {
        CK(launch_ib_front(a, c->cfg.ib_blocks_per_sm, s));     // forces and spread: both in the forces phase
        CK(mark(1));
    } else {
        if (nodes)
            CK(launch_node_force(a, s));
        CK(mark(1));
        if (nodes)
            CK(launch_spread(a, s));
    }
    CK(mark(2));
    if (nodes && c->any_vartau && !split)
        CK(launch_inout(a, s));
    CK(mark(3));
    if (forces_only)
        return IBLB_OK;
    if (split)   // the groups near the band, after the spread
        CK(launch_lb(a, c->storage, c->fbuf[par], c->fbuf[par ^ 1], c->any_vartau, c->cfg, s, a.grp_list,
                     a.grp_cnt, false));
    else
        CK(launch_lb(a, c->storage, c->fbuf[par], c->fbuf[par ^ 1], nodes && c->any_vartau, c->cfg, s));
    CK(mark(4));
    if (nodes && c->fused_ib) {
        CK(launch_ib_back(a, c->n_red_chunks, c->any_volcorr, c->cfg.ib_blocks_per_sm, s));   // advection, volume correction
        CK(mark(5));
    } else {
        if (nodes)
            CK(launch_interp_advect(a, s));
        CK(mark(5));
        if (nodes && c->any_volcorr)
            CK(launch_volume_correction(a, c->n_red_chunks, s));
    }
    if (split)
        CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    CK(mark(6));
    return IBLB_OK;
}

// Capture `nsteps` consecutive steps, the first from buffer parity `par`,
// as one graph.
int capture_steps(iblb_ctx *c, int par, int nsteps, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int r = IBLB_OK;
    for (int i = 0; i < nsteps && r == IBLB_OK; ++i)
        r = enqueue_step(c, par ^ (i & 1), false);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (r != IBLB_OK) {
        if (g)
            cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess)
        return fail(c, IBLB_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(c, IBLB_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return IBLB_OK;
}

int capture_step(iblb_ctx *c, int par)
{
    int r = capture_steps(c, par, 1, &c->gexec[par]);
    if (r == IBLB_OK)
        c->gvalid[par] = true;
    return r;
}

int accumulate_profile(iblb_ctx *c)
{
    if (c->profile == 3) {      // the stream-collide kernel alone
        float ms = 0.f;
        CK(cudaEventSynchronize(c->ph[IBLB_PH_LB + 1]));
        CK(cudaEventElapsedTime(&ms, c->ph[IBLB_PH_LB], c->ph[IBLB_PH_LB + 1]));
        c->ph_ms[IBLB_PH_LB] += ms;
        c->prof_steps++;
        return IBLB_OK;
    }
    CK(cudaEventSynchronize(c->ph[IBLB_NPHASE]));
    for (int k = 0; c->profile == 1 && k < IBLB_NPHASE; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ph[k], c->ph[k + 1]));
        c->ph_ms[k] += ms;
    }
    float tot = 0.f;
    CK(cudaEventElapsedTime(&tot, c->ph[0], c->ph[IBLB_NPHASE]));
    c->step_ms += tot;
    c->prof_steps++;
    return IBLB_OK;
}

int status_code(int flags)
{
    if (flags & ST_TIMEOUT)
        return IBLB_E_TIMEOUT;
    if (flags & (ST_SPREAD_OVF | ST_COL_OVF))
        return IBLB_E_OVERFLOW;
    if (flags & (ST_NAN | ST_JUMP | ST_ESCAPE | ST_BAND_MISS))
        return IBLB_E_UNSTABLE;
    return IBLB_OK;
}

std::string status_text(int flags)
{
    std::string s;
    if (flags & ST_NAN) s += " non-finite node velocity;";
    if (flags & ST_JUMP) s += " a node moved more than 1/2 in one step;";
    if (flags & ST_ESCAPE) s += " a node left the fluid layers;";
    if (flags & ST_SPREAD_OVF) s += " more nodes overlap a band tile than the spread holds;";
    if (flags & ST_COL_OVF) s += " more ray crossings in a column than kept;";
    if (flags & ST_TIMEOUT) s += " a bounded wait gave up;";
    if (flags & ST_BAND_MISS) s += " the band moved by more than one tile row in one step;";
    return s;
}

// read (and optionally clear) the device status of every droplet
int read_status(iblb_ctx *c, bool clear, int *flags_or)
{
    CK(cudaMemcpyAsync(c->h_status, c->A.status, sizeof(int) * 4 * c->ndrops, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int f = 0;
    for (int d = 0; d < c->ndrops; ++d)
        f |= c->h_status[4 * d];
    if (clear && f) {
        for (int d = 0; d < c->ndrops; ++d)
            CK(cudaMemsetAsync(c->A.status + 4 * d, 0, sizeof(int), c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    *flags_or = f;
    return IBLB_OK;
}

// The staging array for one droplet's nodes (x, y, z per node), grown on demand.
int ensure_stage(iblb_ctx *c, int64_t n)
{
    if (n > c->d_stage_n) {
        dfree(c->d_stage);
        c->d_stage = nullptr;
        c->d_stage_n = 0;
        CK(dalloc(&c->d_stage, (size_t)n));
        c->d_stage_n = n;
    }
    return IBLB_OK;
}

int check_k(iblb_ctx *c, int k)
{
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    if (k < 0 || k >= c->ndrops)
        return fail(c, IBLB_E_ARG, "droplet index out of range");
    return IBLB_OK;
}

}  // namespace

extern "C" {

const char *iblb_version(void) { return kVersion; }

const char *iblb_last_error(const iblb_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int iblb_wetting_A(double sigma, double theta_eq_deg, double xi, int n, int m, double *A)
{
    if (!A || !(xi > 0.0) || n <= m)
        return fail(nullptr, IBLB_E_ARG, "iblb_wetting_A: need xi > 0, n > m and an output pointer");
    // eq. A_choice
    *A = sigma * (double)((m - 1) * (n - 1)) / ((double)(n - m) * xi) * (1.0 + cos(theta_eq_deg * M_PI / 180.0));
    return IBLB_OK;
}

int iblb_batch_create(int n, const iblb_lattice_desc *lat, const iblb_physics_desc *phys, void *stream,
                      iblb_ctx **out)
{
    iblb_ctx *c = nullptr;
    if (!out || !lat || !phys || n < 1)
        return fail(nullptr, IBLB_E_ARG, "iblb_batch_create: bad arguments");
    *out = nullptr;
    for (int d = 0; d < n; ++d) {
        std::string why;
        if (!check_desc(lat[d], phys[d], why))
            return fail(nullptr, IBLB_E_ARG, "droplet " + std::to_string(d) + ": " + why);
        if (lat[d].storage != lat[0].storage)
            return fail(nullptr, IBLB_E_ARG, "all droplets of a context need the same storage");
    }
    c = new iblb_ctx();
    c->ndrops = n;
    c->storage = lat[0].storage;
    c->lat.assign(lat, lat + n);
    c->phys.assign(phys, phys + n);
    c->drops.resize(n);
    c->mem.resize(n);
    for (int d = 0; d < n; ++d) {
        memset(&c->drops[d], 0, sizeof(Drop));
        fill_drop_params(c->drops[d], lat[d], phys[d]);
        c->any_vartau |= c->drops[d].vartau != 0;
        c->any_volcorr |= c->drops[d].volcorr != 0;
    }
    c->user = (cudaStream_t)stream;
    int dev = 0;
    auto bad = [&](cudaError_t e, const char *what) {
        std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
        iblb_destroy(c);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? IBLB_E_NOMEM : IBLB_E_CUDA, msg);
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess)
        return bad(e, "cudaGetDevice");
    cudaDeviceGetAttribute(&c->cfg.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bad(e, "cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess)
        return bad(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess)
        return bad(e, "cudaEventCreate");
    for (int k = 0; k <= IBLB_NPHASE; ++k)
        if ((e = cudaEventCreate(&c->ph[k])) != cudaSuccess)
            return bad(e, "cudaEventCreate");
    layout(c);
    Arrays &A = c->A;
    A.ndrops = n;
    const size_t sb = storage_bytes(c->storage);
    const int64_t T = A.total_tiles;
    A.active_cap = (int)T;
    if ((e = cudaMalloc(&c->fbuf[0], sb * Q * A.total_pcells)) != cudaSuccess ||
        (e = cudaMalloc(&c->fbuf[1], sb * Q * A.total_pcells)) != cudaSuccess ||
        (e = dalloc(&A.F, 3 * (size_t)A.total_pcells)) != cudaSuccess ||
        (e = dalloc(&A.U, (size_t)A.total_pcells)) != cudaSuccess ||
        (e = dalloc(&A.tile_gen, (size_t)T)) != cudaSuccess || (e = dalloc(&A.gen, 1)) != cudaSuccess ||
        (e = dalloc(&A.n_active, 2)) != cudaSuccess || (e = dalloc(&A.active, 2 * (size_t)T)) != cudaSuccess ||
        (e = dalloc(&A.bin_cnt, (size_t)T)) != cudaSuccess ||
        (e = dalloc(&A.tile_list, (size_t)T * TILE_CAP)) != cudaSuccess ||
        (e = dalloc(&A.spread_done, 1)) != cudaSuccess || (e = dalloc(&A.bar_count, 1)) != cudaSuccess ||
        (e = dalloc(&A.bar_flag, 1)) != cudaSuccess ||
        (e = dalloc(&A.rowgen, (size_t)A.total_trows)) != cudaSuccess ||
        (e = dalloc(&A.candrow, (size_t)A.total_trows)) != cudaSuccess ||
        (e = dalloc(&A.grp_list, 2 * (size_t)A.total_rows)) != cudaSuccess ||
        (e = dalloc(&A.grp_cnt, 3)) != cudaSuccess || (e = dalloc(&A.split_ok, 1)) != cudaSuccess ||
        (e = dalloc(&A.col_cnt, (size_t)A.total_cols)) != cudaSuccess ||
        (e = dalloc(&A.col_z, (size_t)A.total_cols * MAXC)) != cudaSuccess ||
        (e = dalloc(&A.mass_part, (size_t)c->mass_blocks)) != cudaSuccess ||
        (e = dalloc(&A.status, 4 * (size_t)n)) != cudaSuccess ||
        (e = dalloc(&c->d_mass, (size_t)n)) != cudaSuccess || (e = dalloc(&c->d_drops, (size_t)n)) != cudaSuccess)
        return bad(e, "cudaMalloc");
    if ((e = cudaMallocHost(&c->h_obs, sizeof(double) * (32 + (size_t)n))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming)) != cudaSuccess)
        return bad(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&c->h_status, sizeof(int) * 4 * n)) != cudaSuccess)
        return bad(e, "cudaMallocHost");
    A.drops = c->d_drops;
    cudaStream_t s = c->stream;
    const uint32_t one = 1;
    if ((e = cudaMemsetAsync(A.tile_gen, 0, sizeof(uint32_t) * T, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A.gen, &one, sizeof(one), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.n_active, 0, 2 * sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.spread_done, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.bar_count, 0, sizeof(unsigned), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.bar_flag, 0, sizeof(unsigned), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.rowgen, 0, sizeof(uint32_t) * A.total_trows, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.candrow, 1, A.total_trows, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.grp_cnt, 0, 3 * sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.split_ok, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.bin_cnt, 0, sizeof(int) * T, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.col_cnt, 0, sizeof(int) * A.total_cols, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.status, 0, sizeof(int) * 4 * n, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.F, 0, sizeof(float) * 3 * A.total_pcells, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.U, 0, sizeof(float4) * A.total_pcells, s)) != cudaSuccess ||
        (e = launch_init_populations(A, c->storage, c->fbuf[0], s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->d_drops, c->drops.data(), sizeof(Drop) * n, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return bad(e, "initialisation");
    *out = c;
    return IBLB_OK;
}

int iblb_create(const iblb_lattice_desc *lat, const iblb_physics_desc *phys, void *stream, iblb_ctx **out)
{
    return iblb_batch_create(1, lat, phys, stream, out);
}

void iblb_destroy(iblb_ctx *c)
{
    if (!c)
        return;
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    invalidate_graphs(c);
    free_membrane_arrays(c);
    dfree(c->d_trace);
    Arrays &A = c->A;
    dfree(c->fbuf[0]);
    dfree(c->fbuf[1]);
    dfree(A.F);
    dfree(A.U);
    dfree(A.tile_gen);
    dfree(A.gen);
    dfree(A.n_active);
    dfree(A.active);
    dfree(A.bin_cnt);
    dfree(A.tile_list);
    dfree(A.spread_done);
    dfree(A.bar_count);
    dfree(A.bar_flag);
    dfree(A.rowgen);
    dfree(A.candrow);
    dfree(A.grp_list);
    dfree(A.grp_cnt);
    dfree(A.split_ok);
    dfree(A.col_cnt);
    dfree(A.col_z);
    dfree(A.mass_part);
    dfree(A.status);
    dfree(c->d_mass);
    dfree(c->d_drops);
    dfree(c->obs_scr);
    if (c->h_status)
        cudaFreeHost(c->h_status);
    if (c->h_obs)
        cudaFreeHost(c->h_obs);
    if (c->ev_copy)
        cudaEventDestroy(c->ev_copy);
    dfree(c->d_stage);
    for (int k = 0; k <= IBLB_NPHASE; ++k)
        if (c->ph[k])
            cudaEventDestroy(c->ph[k]);
    if (c->ev_in)
        cudaEventDestroy(c->ev_in);
    if (c->ev_out)
        cudaEventDestroy(c->ev_out);
    if (c->ev_fork)
        cudaEventDestroy(c->ev_fork);
    if (c->ev_join)
        cudaEventDestroy(c->ev_join);
    if (c->side)
        cudaStreamDestroy(c->side);
    if (c->stream)
        cudaStreamDestroy(c->stream);
    delete c;
}

int iblb_info(const iblb_ctx *ctx, int k, int *n_drops, int64_t *cells, int *n_nodes, int *n_tri)
{
    iblb_ctx *c = const_cast<iblb_ctx *>(ctx);
    int r = check_k(c, k);
    if (r)
        return r;
    if (n_drops)
        *n_drops = c->ndrops;
    if (cells)
        *cells = c->drops[k].cells;
    if (n_nodes)
        *n_nodes = c->mem[k].set ? (int)(c->mem[k].xyz.size() / 3) : 0;
    if (n_tri)
        *n_tri = c->mem[k].set ? (int)(c->mem[k].tri.size() / 3) : 0;
    return IBLB_OK;
}

int iblb_check_mesh(const double *xyz, int n_nodes, const int32_t *tri, int n_tri, double *volume)
{
    if (!xyz || !tri)
        return fail(nullptr, IBLB_E_ARG, "iblb_check_mesh: null mesh arrays");
    std::string why;
    double V = 0.0;
    if (!validate_mesh(xyz, n_nodes, tri, n_tri, why, &V))
        return fail(nullptr, IBLB_E_MESH, why);
    if (volume)
        *volume = V;
    return IBLB_OK;
}

int iblb_set_membrane(iblb_ctx *c, int k, const double *xyz, int n_nodes, const int32_t *tri, int n_tri)
{
    Trace trace_("iblb_set_membrane");
    int r = check_k(c, k);
    if (r)
        return r;
    if (!xyz || !tri)
        return fail(c, IBLB_E_ARG, "null mesh arrays");
    std::string why;
    double V = 0.0;
    if (!validate_mesh(xyz, n_nodes, tri, n_tri, why, &V))
        return fail(c, IBLB_E_MESH, why);
    if (c->A.total_nodes && (r = download_nodes(c)))   // keep the other droplets' current state
        return r;
    Membrane &M = c->mem[k];
    M.xyz.assign(xyz, xyz + 3 * (size_t)n_nodes);
    M.ref = M.xyz;
    M.tri.assign(tri, tri + 3 * (size_t)n_tri);
    M.set = true;
    M.V0 = V;
    std::fill(M.corr, M.corr + NRED, 0.0);   // no volume correction pending
    M.corr[0] = 1.0;
    c->mem_dirty = true;
    return rebuild_membranes(c);
}

int iblb_set_nodes(iblb_ctx *c, int k, const double *xyz)
{
    int r = check_k(c, k);
    if (r || (r = ensure_ready(c)))
        return r;
    const Drop &D = c->drops[k];
    if (!D.nnodes)
        return fail(c, IBLB_E_STATE, "droplet has no membrane");
    Entered entered_(c);
    if ((r = ensure_stage(c, 3 * (int64_t)D.nnodes)))
        return r;
    // one copy of the caller's x, y, z per node; the split into the position
    // planes and their FP32 pairs runs on the device
    CK(cudaMemcpyAsync(c->d_stage, xyz, sizeof(double) * 3 * D.nnodes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaEventRecord(c->ev_copy, c->stream));
    CK(launch_set_nodes(c->A, c->d_stage, D.node0, D.nnodes, k, c->stream));
    // the given positions are final: no volume correction pending on them
    c->mem[k].corr[5] = 0.0;
    CK(cudaEventSynchronize(c->ev_copy));   // the caller may reuse xyz
    return IBLB_OK;
}

int iblb_get_nodes(iblb_ctx *c, int k, double *xyz)
{
    int r = check_k(c, k);
    if (r || (r = ensure_ready(c)))
        return r;
    const Drop &D = c->drops[k];
    if (!D.nnodes)
        return fail(c, IBLB_E_STATE, "droplet has no membrane");
    Entered entered_(c);
    if ((r = ensure_stage(c, 3 * (int64_t)D.nnodes)))
        return r;
    // the positions with the pending volume correction, interleaved on the device
    CK(launch_corrected_positions(c->A, c->stream, c->d_stage, D.node0, D.nnodes));
    CK(cudaMemcpyAsync(xyz, c->d_stage, sizeof(double) * 3 * D.nnodes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IBLB_OK;
}

// temporary device buffer for one transfer
struct Tmp {
    void *p = nullptr;
    ~Tmp() { dfree(p); }
};

int iblb_set_populations(iblb_ctx *c, int k, const double *f)
{
    int r = check_k(c, k);
    if (r)
        return r;
    const Drop &D = c->drops[k];
    Tmp t;
    CK(cudaMalloc(&t.p, sizeof(double) * Q * D.cells));
    Entered entered_(c);
    CK(cudaMemcpyAsync(t.p, f, sizeof(double) * Q * D.cells, cudaMemcpyHostToDevice, c->stream));
    CK(launch_import_populations(c->A, k, c->storage, c->fbuf[c->cur], (const double *)t.p, D.cells, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IBLB_OK;
}

int iblb_get_populations(iblb_ctx *c, int k, double *f)
{
    int r = check_k(c, k);
    if (r)
        return r;
    const Drop &D = c->drops[k];
    Tmp t;
    CK(cudaMalloc(&t.p, sizeof(double) * Q * D.cells));
    Entered entered_(c);
    CK(launch_export_populations(c->A, k, c->storage, c->fbuf[c->cur], (double *)t.p, D.cells, c->stream));
    CK(cudaMemcpyAsync(f, t.p, sizeof(double) * Q * D.cells, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IBLB_OK;
}

int iblb_get_macros(iblb_ctx *c, int k, double *rho, double *u)
{
    int r = check_k(c, k);
    if (r)
        return r;
    const Drop &D = c->drops[k];
    Tmp t;
    CK(cudaMalloc(&t.p, sizeof(double) * 4 * D.cells));
    double *dr = (double *)t.p, *du = dr + D.cells;
    Entered entered_(c);
    CK(launch_export_macros(c->A, k, c->storage, c->fbuf[c->cur], dr, du, D.cells, c->stream));
    CK(cudaMemcpyAsync(rho, dr, sizeof(double) * D.cells, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(u, du, sizeof(double) * 3 * D.cells, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IBLB_OK;
}

int iblb_compute_forces(iblb_ctx *c)
{
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    int r = ensure_ready(c);
    if (r)
        return r;
    const int prof = c->profile;
    c->profile = 0;
    Entered entered_(c);
    r = enqueue_step(c, c->cur, true);
    c->profile = prof;
    if (r)
        return r;
    CK(cudaStreamSynchronize(c->stream));
    int flags = 0;
    if ((r = read_status(c, false, &flags)))
        return r;
    if (status_code(flags))
        return fail(c, status_code(flags), "device status:" + status_text(flags));
    return IBLB_OK;
}

int iblb_get_node_forces(iblb_ctx *c, int k, double *phi)
{
    int r = check_k(c, k);
    if (r || (r = ensure_ready(c)))
        return r;
    const Drop &D = c->drops[k];
    if (!D.nnodes)
        return fail(c, IBLB_E_STATE, "droplet has no membrane");
    std::vector<NodeRec> rec(D.nnodes);
    Entered entered_(c);
    CK(cudaMemcpyAsync(rec.data(), c->A.rec + D.node0, sizeof(NodeRec) * D.nnodes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int j = 0; j < D.nnodes; ++j)
        for (int e = 0; e < 3; ++e)
            phi[3 * j + e] = rec[j].phi[e];
    return IBLB_OK;
}

int iblb_get_force_density(iblb_ctx *c, int k, double *F)
{
    int r = check_k(c, k);
    if (r)
        return r;
    const Drop &D = c->drops[k];
    Tmp t;
    CK(cudaMalloc(&t.p, sizeof(double) * 3 * D.cells));
    Entered entered_(c);
    CK(launch_export_force(c->A, k, (double *)t.p, D.cells, c->stream));
    CK(cudaMemcpyAsync(F, t.p, sizeof(double) * 3 * D.cells, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IBLB_OK;
}

int iblb_get_inside(iblb_ctx *c, int k, uint8_t *inside)
{
    int r = check_k(c, k);
    if (r)
        return r;
    const Drop &D = c->drops[k];
    Tmp t;
    CK(cudaMalloc(&t.p, D.cells));
    Entered entered_(c);
    CK(launch_export_inside(c->A, k, (uint8_t *)t.p, D.cells, c->stream));
    CK(cudaMemcpyAsync(inside, t.p, D.cells, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IBLB_OK;
}

int iblb_step(iblb_ctx *c, int nsteps)
{
    Trace trace_("iblb_step");
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    if (nsteps < 0)
        return fail(c, IBLB_E_ARG, "nsteps < 0");
    int r = ensure_ready(c);
    if (r)
        return r;
    Entered entered_(c);
    // whole chunks of K steps as one graph each (not while profiling, which
    // times every step from the host)
    const int K = c->graph_chunk;
    while (c->graphs && !c->profile && K > 1 && nsteps >= K) {
        const int par = c->cur;
        if (!c->gchunk[par] && (r = capture_steps(c, par, K, &c->gchunk[par])))
            return r;
        CK(cudaGraphLaunch(c->gchunk[par], c->stream));
        c->cur ^= K & 1;
        c->step_count += K;
        nsteps -= K;
    }
    for (int i = 0; i < nsteps; ++i) {
        const int par = c->cur;
        if (c->graphs) {
            if (!c->gvalid[par] && (r = capture_step(c, par)))
                return r;
            CK(cudaGraphLaunch(c->gexec[par], c->stream));
        } else if ((r = enqueue_step(c, par, false))) {
            return r;
        }
        c->cur ^= 1;
        c->step_count++;
        if (c->profile && (r = accumulate_profile(c)))
            return r;
    }
    return IBLB_OK;
}

int iblb_trace_step(iblb_ctx *c, double *out)
{
    Trace trace_("iblb_trace_step");
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    if (!out)
        return fail(c, IBLB_E_ARG, "null output");
    int r = ensure_ready(c);
    if (r)
        return r;
    Entered entered_(c);
    const size_t n = (size_t)(TRACE_KERNELS + 1) * TRACE_WARPS;
    if (!c->d_trace)
        CK(dalloc(&c->d_trace, n));
    CK(cudaMemsetAsync(c->d_trace, 0, n * sizeof(unsigned long long), c->stream));
    const int prof = c->profile;
    c->profile = 0;
    set_trace_ib(c->d_trace);
    set_trace_lb(c->d_trace);
    r = enqueue_step(c, c->cur, false);
    const cudaError_t em = r ? cudaSuccess : launch_trace_marker(c->A, c->d_trace, c->stream);
    set_trace_ib(nullptr);
    set_trace_lb(nullptr);
    c->profile = prof;
    if (r)
        return r;
    CK(em);
    c->cur ^= 1;
    c->step_count++;
    std::vector<unsigned long long> h(n);
    CK(cudaMemcpyAsync(h.data(), c->d_trace, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // per kernel (and the marker): first, median and last warp start
    double first[TRACE_KERNELS + 1], med[TRACE_KERNELS + 1], last[TRACE_KERNELS + 1];
    int warps[TRACE_KERNELS + 1];
    unsigned long long t0 = ~0ull;
    for (size_t i = 0; i < n; ++i)
        if (h[i])
            t0 = std::min(t0, h[i]);
    for (int k = 0; k <= TRACE_KERNELS; ++k) {
        std::vector<unsigned long long> v;
        for (int w = 0; w < TRACE_WARPS; ++w)
            if (h[(size_t)k * TRACE_WARPS + w])
                v.push_back(h[(size_t)k * TRACE_WARPS + w]);
        warps[k] = (int)v.size();
        if (v.empty()) {
            first[k] = med[k] = last[k] = NAN;
            continue;
        }
        std::sort(v.begin(), v.end());
        first[k] = (double)(v.front() - t0) * 1e-3;
        med[k] = (double)(v[v.size() / 2] - t0) * 1e-3;
        last[k] = (double)(v.back() - t0) * 1e-3;
    }
    for (int k = 0; k < TRACE_KERNELS; ++k) {
        double *o = out + 5 * k;
        o[0] = first[k];
        o[1] = med[k];
        o[2] = last[k];
        o[3] = NAN;             // end: the first start of the next kernel that ran
        for (int m = k + 1; m <= TRACE_KERNELS && warps[k]; ++m)
            if (warps[m]) {
                o[3] = first[m];
                break;
            }
        o[4] = (double)warps[k];
    }
    return IBLB_OK;
}

int iblb_sync(iblb_ctx *c)
{
    Trace trace_("iblb_sync");
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    CK(cudaStreamSynchronize(c->stream));
    int flags = 0, r = read_status(c, true, &flags);
    if (r)
        return r;
    if (status_code(flags))
        return fail(c, status_code(flags), "device status:" + status_text(flags));
    return IBLB_OK;
}

// mesh observables and status of droplet k into out (the mass is filled by
// the caller; the corrected positions are in c->A.p*); the observation
// scratch is kept in the context
// Enqueue the mesh observation of droplet k (kernels and a copy of the raw
// results to c->h_obs); observe_mesh_finish fills out once the stream has
// passed them (and c->h_status was refreshed with them).
int observe_mesh_enqueue(iblb_ctx *c, int k, double zcut_frac, double eps_flat)
{
    const Drop &D = c->drops[k];
    if (!D.nnodes)
        return IBLB_OK;
    const int64_t need = observe_scratch_doubles(D.nnodes, D.ntri);
    if (need > c->obs_scr_n) {
        dfree(c->obs_scr);
        c->obs_scr = nullptr;
        c->obs_scr_n = 0;
        CK(dalloc(&c->obs_scr, (size_t)need));
        c->obs_scr_n = need;
    }
    CK(enqueue_observe(c->A.px, c->A.py, c->A.pz, c->A.clamped, c->A.tri + 3 * (int64_t)D.tri0, D.ntri, D.node0,
                       D.nnodes, D.R0, zcut_frac, eps_flat, c->obs_scr, c->h_obs, c->stream));
    return IBLB_OK;
}

void observe_mesh_finish(iblb_ctx *c, int k, iblb_obs *out)
{
    const Drop &D = c->drops[k];
    if (D.nnodes) {
        double h[14];
        finish_observe(c->h_obs, D.R0, h);
        out->volume = h[0];
        out->area = h[1];
        out->centroid[0] = h[2];
        out->centroid[1] = h[3];
        out->centroid[2] = h[4];
        out->zmin = h[5];
        out->zmax = h[6];
        out->theta_R0_deg = h[7];
        out->theta_RV_deg = h[8];
        out->rc_cut = h[9];
        out->rc_flat = h[10];
        out->n_cut = h[11];
        out->chi_flat = h[12];
        out->clamped = (int)h[13];
    }
    // this droplet's flags; a bounded-wait timeout is recorded on droplet 0
    // and concerns every droplet
    out->status = status_code(c->h_status[4 * k] | (c->h_status[0] & ST_TIMEOUT));
}

int iblb_observe(iblb_ctx *c, int k, double zcut_frac, double eps_flat, iblb_obs *out)
{
    Trace trace_("iblb_observe");
    int r = check_k(c, k);
    if (r || (r = ensure_ready(c)))
        return r;
    if (!out)
        return fail(c, IBLB_E_ARG, "null output");
    memset(out, 0, sizeof(*out));
    Entered entered_(c);
    // everything enqueued, one synchronisation: the mass, the corrected
    // positions and the mesh passes, then the copies of their results and of
    // the status words to pinned host memory
    CK(launch_mass(c->A, c->storage, c->fbuf[c->cur], c->d_mass, c->mass_blocks, c->stream));
    CK(launch_corrected_positions(c->A, c->stream));
    if ((r = observe_mesh_enqueue(c, k, zcut_frac, eps_flat)))
        return r;
    CK(cudaMemcpyAsync(c->h_obs + 32 + k, c->d_mass + k, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->h_status, c->A.status, sizeof(int) * 4 * c->ndrops, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out->mass = c->h_obs[32 + k];
    observe_mesh_finish(c, k, out);
    return IBLB_OK;
}

int iblb_observe_all(iblb_ctx *c, double zcut_frac, double eps_flat, iblb_obs *out)
{
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    int r = ensure_ready(c);
    if (r)
        return r;
    if (!out)
        return fail(c, IBLB_E_ARG, "null output");
    memset(out, 0, sizeof(*out) * (size_t)c->ndrops);
    Entered entered_(c);
    CK(launch_mass(c->A, c->storage, c->fbuf[c->cur], c->d_mass, c->mass_blocks, c->stream));
    CK(cudaMemcpyAsync(c->h_obs + 32, c->d_mass, sizeof(double) * c->ndrops, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->h_status, c->A.status, sizeof(int) * 4 * c->ndrops, cudaMemcpyDeviceToHost, c->stream));
    CK(launch_corrected_positions(c->A, c->stream));
    for (int k = 0; k < c->ndrops; ++k) {   // one droplet at a time through the shared scratch
        if ((r = observe_mesh_enqueue(c, k, zcut_frac, eps_flat)))
            return r;
        CK(cudaStreamSynchronize(c->stream));
        out[k].mass = c->h_obs[32 + k];
        observe_mesh_finish(c, k, &out[k]);
    }
    return IBLB_OK;
}

int iblb_set_option(iblb_ctx *c, int option, int value)
{
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    switch (option) {
    case IBLB_OPT_GRAPHS:
        c->graphs = value != 0;
        return IBLB_OK;
    case IBLB_OPT_PROFILE:
        if (value < 0 || value > 3)
            return fail(c, IBLB_E_ARG, "profile mode must be 0, 1, 2 or 3");
        if (c->profile != value)
            invalidate_graphs(c);
        c->profile = value;
        return IBLB_OK;
    case IBLB_OPT_LB_BLOCKS_PER_SM:
        if (value < 0 || value > 8)
            return fail(c, IBLB_E_ARG, "resident blocks per SM must be in [0, 8]");
        c->cfg.lb_blocks_per_sm = value;
        invalidate_graphs(c);
        return IBLB_OK;
    case IBLB_OPT_LB_GROUP_CELLS: {
        if (value < 0 || value > 16384)
            return fail(c, IBLB_E_ARG, "cells per group must be in [0, 16384]");
        int r = ensure_ready(c);
        if (r)
            return r;
        c->cfg.lb_group_cells = value;
        layout(c);
        invalidate_graphs(c);
        return upload_drops(c);
    }
    case IBLB_OPT_LB_ROW_MULT: {
        if (value == 0)
            value = 1;
        if (value < 1 || value > 4)
            return fail(c, IBLB_E_ARG, "row multiplier must be in [1, 4]");
        int r = ensure_ready(c);
        if (r)
            return r;
        c->cfg.lb_row_mult = value;
        c->cfg.lb_group_cells = 0;             // the multiplier takes over
        layout(c);
        invalidate_graphs(c);
        return upload_drops(c);
    }
    case IBLB_OPT_FUSED_IB:
        c->fused_ib = value != 0;
        invalidate_graphs(c);
        return IBLB_OK;
    case IBLB_OPT_GRAPH_CHUNK:
        if (value < 1 || value > 64)
            return fail(c, IBLB_E_ARG, "steps per graph must be in [1, 64]");
        if (c->graph_chunk != value)
            invalidate_graphs(c);
        c->graph_chunk = value;
        return IBLB_OK;
    case IBLB_OPT_PDL:
        c->pdl = value != 0;
        invalidate_graphs(c);
        return IBLB_OK;
    case IBLB_OPT_SPLIT_LB:
        c->split_lb = value != 0;
        invalidate_graphs(c);
        return IBLB_OK;
    case IBLB_OPT_LB_FAR_BLOCKS_PER_SM:
        if (value < 0 || value > 8)
            return fail(c, IBLB_E_ARG, "blocks per SM must be in [0, 8]");
        c->lb_far_blocks_per_sm = value;
        invalidate_graphs(c);
        return IBLB_OK;
    case IBLB_OPT_IB_BLOCKS_PER_SM:
        if (value < 0 || value > 8)
            return fail(c, IBLB_E_ARG, "membrane blocks per SM must be in [0, 8]");
        c->cfg.ib_blocks_per_sm = value;
        invalidate_graphs(c);
        return IBLB_OK;
    case IBLB_OPT_LB_STAGES:
        if (value < 2 || value > 8)
            return fail(c, IBLB_E_ARG, "pipeline stages must be in [2, 8]");
        c->cfg.lb_stages = value;
        fit_stages(c);
        invalidate_graphs(c);
        return IBLB_OK;
    }
    return fail(c, IBLB_E_ARG, "unknown option");
}

int iblb_get_profile(iblb_ctx *c, double *phase_ms, double *step_ms, int64_t *steps)
{
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    if (phase_ms)
        for (int k = 0; k < IBLB_NPHASE; ++k)
            phase_ms[k] = c->ph_ms[k];
    if (step_ms)
        *step_ms = c->step_ms;
    if (steps)
        *steps = c->prof_steps;
    return IBLB_OK;
}

int iblb_reset_profile(iblb_ctx *c)
{
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    for (int k = 0; k < IBLB_NPHASE; ++k)
        c->ph_ms[k] = 0.0;
    c->step_ms = 0.0;
    c->prof_steps = 0;
    return IBLB_OK;
}

int iblb_autotune(iblb_ctx *c, const char *cache_path)
{
    Trace trace_("iblb_autotune");
    if (!c)
        return fail(nullptr, IBLB_E_ARG, "null context");
    int r = ensure_ready(c);
    if (r)
        return r;
    char key[160];
    snprintf(key, sizeof(key), "storage=%d cells=%lld drops=%d vartau=%d", c->storage,
             (long long)c->A.total_cells, c->ndrops, (int)c->any_vartau);
    if (cache_path) {
        FILE *fp = fopen(cache_path, "r");
        if (fp) {
            char line[256];
            while (fgets(line, sizeof(line), fp)) {
                int bps = 0, mult = 0, ns = 2, cells = 0;
                const char *bar = strchr(line, '|');
                if (bar && (size_t)(bar - line) == strlen(key) && !strncmp(line, key, strlen(key)) &&
                    sscanf(bar + 1, "%d %d %d %d", &bps, &mult, &ns, &cells) == 4) {
                    fclose(fp);
                    if ((r = iblb_set_option(c, IBLB_OPT_LB_BLOCKS_PER_SM, bps)) ||
                        (r = iblb_set_option(c, IBLB_OPT_LB_STAGES, ns)) ||
                        (r = iblb_set_option(c, IBLB_OPT_LB_ROW_MULT, mult)))
                        return r;
                    return iblb_set_option(c, IBLB_OPT_LB_GROUP_CELLS, cells);
                }
            }
            fclose(fp);
        }
    }
    // time the stream-collide kernel alone from the current buffer into the
    // spare one: the current state is left untouched
    const int bpsm[2] = {0, 1};
    float best = 1e30f;
    int bb = c->cfg.lb_blocks_per_sm, bm = c->cfg.lb_row_mult, bcells = c->cfg.lb_group_cells;
    int dev = 0, smem_max = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    struct Events {   // destroyed on every way out
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events()
        {
            for (cudaEvent_t x : e)
                if (x)
                    cudaEventDestroy(x);
        }
    } ev;
    CK(cudaEventCreate(&ev.e[0]));
    CK(cudaEventCreate(&ev.e[1]));
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    Entered entered_(c);
    int bs = c->cfg.lb_stages;
    // group sizes of 256 .. 1024 cells in steps of 128 (whole rows), with
    // every pipeline depth and both residencies whose stages fit
    for (int cells = 256; cells <= 1024; cells += 128)
        for (int bi = 0; bi < 2; ++bi)
            for (int ns = 2; ns <= 8; ++ns) {
                c->cfg.lb_blocks_per_sm = bpsm[bi];
                c->cfg.lb_group_cells = cells;
                c->cfg.lb_stages = ns;
                layout(c);
                if (ns * (int64_t)c->A.lb_stage_bytes + 1024 > smem_max)
                    continue;                  // these stages do not fit
                if ((r = upload_drops(c)))
                    return r;
                const bool vt = c->A.total_nodes > 0 && c->any_vartau;
                for (int w = 0; w < 2; ++w)
                    CK(launch_lb(c->A, c->storage, c->fbuf[c->cur], c->fbuf[c->cur ^ 1], vt, c->cfg, c->stream));
                CK(cudaEventRecord(e0, c->stream));
                for (int w = 0; w < 5; ++w)
                    CK(launch_lb(c->A, c->storage, c->fbuf[c->cur], c->fbuf[c->cur ^ 1], vt, c->cfg, c->stream));
                CK(cudaEventRecord(e1, c->stream));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    bb = bpsm[bi];
                    bcells = cells;
                    bs = ns;
                }
            }
    c->cfg.lb_blocks_per_sm = bb;
    c->cfg.lb_row_mult = bm;
    c->cfg.lb_group_cells = bcells;
    c->cfg.lb_stages = bs;
    layout(c);
    invalidate_graphs(c);
    if ((r = upload_drops(c)))
        return r;
    if (cache_path) {
        FILE *fp = fopen(cache_path, "a");
        if (fp) {
            fprintf(fp, "%s|%d %d %d %d\n", key, bb, bm, bs, bcells);
            fclose(fp);
        }
    }
    return IBLB_OK;
}

int iblb_save(iblb_ctx *c, const char *path)
{
    if (!c || !path)
        return fail(c, IBLB_E_ARG, "null argument");
    int r = ensure_ready(c);
    if (r || (r = download_nodes(c)))
        return r;
    FILE *fp = fopen(path, "wb");
    if (!fp)
        return fail(c, IBLB_E_IO, std::string("cannot open ") + path);
    const size_t sb = storage_bytes(c->storage);
    std::vector<char> buf;
    bool ok = true;
    const char magic[8] = {'I', 'B', 'L', 'B', 'C', 'K', '0', '2'};
    ok &= fwrite(magic, 8, 1, fp) == 1;
    const int64_t hdr[4] = {c->ndrops, c->storage, c->step_count, c->A.total_cells};
    ok &= fwrite(hdr, sizeof(hdr), 1, fp) == 1;
    CK(cudaStreamSynchronize(c->stream));
    for (int d = 0; d < c->ndrops && ok; ++d) {
        const Drop &D = c->drops[d];
        const int64_t dh[3] = {D.cells, D.nnodes, D.ntri};
        ok &= fwrite(dh, sizeof(dh), 1, fp) == 1;
        buf.resize(sb * Q * D.pcells);
        CK(cudaMemcpy(buf.data(), (char *)c->fbuf[c->cur] + sb * Q * D.pcell0, buf.size(), cudaMemcpyDeviceToHost));
        ok &= fwrite(buf.data(), buf.size(), 1, fp) == 1;
        if (D.nnodes) {
            ok &= fwrite(c->mem[d].xyz.data(), sizeof(double) * 3 * D.nnodes, 1, fp) == 1;
            ok &= fwrite(&c->mem[d].V0, sizeof(double), 1, fp) == 1;
            ok &= fwrite(c->mem[d].corr, sizeof(double) * NRED, 1, fp) == 1;
        }
    }
    ok &= fclose(fp) == 0;
    return ok ? IBLB_OK : fail(c, IBLB_E_IO, "write failed");
}

int iblb_load(iblb_ctx *c, const char *path)
{
    if (!c || !path)
        return fail(c, IBLB_E_ARG, "null argument");
    int r = ensure_ready(c);
    if (r)
        return r;
    FILE *fp = fopen(path, "rb");
    if (!fp)
        return fail(c, IBLB_E_IO, std::string("cannot open ") + path);
    const size_t sb = storage_bytes(c->storage);
    char magic[8];
    int64_t hdr[4];
    bool ok = fread(magic, 8, 1, fp) == 1 && !memcmp(magic, "IBLBCK02", 8) && fread(hdr, sizeof(hdr), 1, fp) == 1 &&
              hdr[0] == c->ndrops && hdr[1] == c->storage && hdr[3] == c->A.total_cells;
    std::vector<char> buf;
    CK(cudaStreamSynchronize(c->stream));
    for (int d = 0; d < c->ndrops && ok; ++d) {
        Drop &D = c->drops[d];
        int64_t dh[3];
        ok &= fread(dh, sizeof(dh), 1, fp) == 1 && dh[0] == D.cells && dh[1] == D.nnodes && dh[2] == D.ntri;
        if (!ok)
            break;
        buf.resize(sb * Q * D.pcells);
        ok &= fread(buf.data(), buf.size(), 1, fp) == 1;
        if (!ok)
            break;
        CK(cudaMemcpy((char *)c->fbuf[c->cur] + sb * Q * D.pcell0, buf.data(), buf.size(), cudaMemcpyHostToDevice));
        if (D.nnodes) {
            std::vector<double> xyz(3 * (size_t)D.nnodes);
            double V0 = 0.0, corr[NRED];
            ok &= fread(xyz.data(), sizeof(double) * xyz.size(), 1, fp) == 1 && fread(&V0, sizeof(double), 1, fp) == 1 &&
                  fread(corr, sizeof(double) * NRED, 1, fp) == 1;
            if (!ok)
                break;
            c->mem[d].xyz = xyz;
            c->mem[d].V0 = V0;
            memcpy(c->mem[d].corr, corr, sizeof(corr));
        }
    }
    fclose(fp);
    if (!ok)
        return fail(c, IBLB_E_IO, "checkpoint does not match this context or is truncated");
    c->step_count = hdr[2];
    c->mem_dirty = true;
    return rebuild_membranes(c);
}

int iblb_mesh_observe_dev(const double *d_xyz, int n_nodes, const int32_t *d_tri, int n_tri, double R0,
                          double zcut_frac, double eps_flat, void *stream, double *out)
{
    iblb_ctx *c = nullptr;
    if (!d_xyz || !d_tri || !out || n_nodes < 1 || n_tri < 1 || !(R0 > 0.0))
        return fail(nullptr, IBLB_E_ARG, "iblb_mesh_observe_dev: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    double *scr = nullptr;
    CK(cudaMallocAsync((void **)&scr, sizeof(double) * observe_scratch_doubles(n_nodes, n_tri), s));
    cudaError_t e = launch_observe_view(d_xyz, d_xyz + 1, d_xyz + 2, 3, d_tri, n_tri, 0, n_nodes, R0, zcut_frac,
                                        eps_flat, scr, out, s);
    cudaFreeAsync(scr, s);
    CK(e);
    CK(cudaStreamSynchronize(s));
    return IBLB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Mesh observables with their scratch in a fixed device array.
//
// iblb_mesh_observe_dev takes its scratch from cudaMallocAsync.  Some callers
// cannot allocate device memory at the moment they want the observables: a
// monitor that samples a droplet while a caching allocator (PyTorch's, for
// instance) has claimed all free device memory, where any further allocation
// fails with out-of-memory; or a handler that runs because an allocation just
// failed and wants to record the droplet's state before giving up.  This
// variant runs the same kernels on a statically sized __device__ array.  The
// array holds the scratch of kNoAllocMaxChunks reduction chunks (53.6 KB of
// doubles), the most any mesh uses; meshes are accepted up to 1,048,576
// faces and 524,288 nodes (RED_FACES faces and RED_NODES nodes a chunk at
// most).
//
// Set-up.  The first call made in a CUDA context (normally a device's primary
// context) loads the library's code for that context, looks up the array's
// device address with cudaGetSymbolAddress and checks the result.  Module
// loading is lazy by default and a load allocates device memory, so the
// set-up loads the array's module and the observation kernels at once; after
// it, calls on that context allocate nothing.  The address is kept per device
// together with the identity of the context it was taken in: if the context
// changes (after cudaDeviceReset, or with another context made current), the
// set-up runs again instead of reusing an address of a context that is gone.
// So make one call per device early, while memory is still free, and before
// any stream capture.
//
// Nothing in the array needs to start at zero: every element the kernels read
// is written earlier in the same call.  The array is one per device and the
// call is not reentrant: two calls in flight at once on the same device (from
// two host threads, or on two streams) share it and race.  A call returns only
// after its stream has drained, so calls made one after another are safe.
namespace {
constexpr int kNoAllocMaxChunks = 512;
constexpr int kNoAllocMaxFaces = kNoAllocMaxChunks * RED_FACES;
constexpr int kNoAllocMaxNodes = kNoAllocMaxChunks * RED_NODES;
constexpr int64_t kNoAllocScratch = (int64_t)NRED * kNoAllocMaxChunks + 32 + 5 * (int64_t)kNoAllocMaxChunks + 8;
constexpr int kNoAllocMaxDevices = 256;
struct NoAllocSlot {
    unsigned long long ctx_id = 0;   // 0: no set-up yet (context ids start at 1)
    double *ptr = nullptr;
};
std::mutex g_noalloc_mu;
NoAllocSlot g_noalloc[kNoAllocMaxDevices];

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// the unique id of the calling thread's current context (0 if none), through
// the driver entry points that the runtime hands out
cudaError_t current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    *id = 0;
    if (!get_current || !get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess)
            return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        get_current = (CtxGetCurrentFn)f1;
        get_id = (CtxGetIdFn)f2;
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0)
        return cudaErrorDeviceUninitialized;
    if (ctx && get_id(ctx, id) != 0)
        return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}
}  // namespace

static __device__ __align__(256) double g_observe_scratch[kNoAllocScratch];

namespace {
// the set-up described above, for the current device and context
cudaError_t noalloc_scratch(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess)
        return e;
    NoAllocSlot &slot = g_noalloc[dev];
    if (id == 0 || slot.ctx_id != id) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_observe_scratch);   // makes the primary context current if none is
        if (e != cudaSuccess)
            return e;
        if ((e = preload_observe_kernels()) != cudaSuccess)
            return e;
        if ((e = current_context_id(&id)) != cudaSuccess)
            return e;
        if (id == 0)
            return cudaErrorDeviceUninitialized;
        slot.ctx_id = id;
        slot.ptr = p;
    }
    *out = slot.ptr;
    return cudaSuccess;
}
}  // namespace

extern "C" {

int iblb_mesh_observe_dev_noalloc(const double *d_xyz, int n_nodes, const int32_t *d_tri, int n_tri, double R0,
                                  double zcut_frac, double eps_flat, void *stream, double *out)
{
    iblb_ctx *c = nullptr;
    if (!d_xyz || !d_tri || !out || n_nodes < 1 || n_tri < 1 || !(R0 > 0.0))
        return fail(nullptr, IBLB_E_ARG, "iblb_mesh_observe_dev_noalloc: bad arguments");
    if (n_tri > kNoAllocMaxFaces || n_nodes > kNoAllocMaxNodes ||
        observe_scratch_doubles(n_nodes, n_tri) > kNoAllocScratch)
        return fail(nullptr, IBLB_E_ARG,
                    "iblb_mesh_observe_dev_noalloc: mesh too large for the static scratch (at most " +
                        std::to_string(kNoAllocMaxFaces) + " faces and " + std::to_string(kNoAllocMaxNodes) +
                        " nodes); use iblb_mesh_observe_dev");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(nullptr, IBLB_E_ARG, "iblb_mesh_observe_dev_noalloc: device ordinal out of range");
    double *scr = nullptr;
    CK(noalloc_scratch(dev, &scr));
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_observe_view(d_xyz, d_xyz + 1, d_xyz + 2, 3, d_tri, n_tri, 0, n_nodes, R0, zcut_frac, eps_flat, scr,
                           out, s));
    CK(cudaStreamSynchronize(s));
    return IBLB_OK;
}

}  // extern "C"
