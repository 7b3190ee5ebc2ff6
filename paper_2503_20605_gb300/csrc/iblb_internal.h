// iblb_internal.h -- data layout shared by the host code and the kernels of
// libiblb.  Every kernel works over a table of droplets (a context with one
// droplet is a table of length one), so the batched path and the single
// path execute the same arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace iblb {

constexpr int Q = 19;
constexpr int TILE = 4;            // band tiles are 4x4x4 fluid cells
constexpr int TILE_CELLS = 64;
constexpr int MAXC = 16;           // ray crossings kept per lattice column
constexpr int TILE_CAP = 512;      // nodes whose kernel support may touch one tile
constexpr int RED_FACES = 2048;    // at most this many faces and nodes per chunk of the observation
constexpr int RED_NODES = 1024;    // reductions within the allocation-free call's limit (512 chunks)
constexpr int MASS_CELLS_PER_BLOCK = 1024;   // cells per block of the lattice-mass reduction
constexpr int VC_ITEMS = 128;      // faces (and nodes) per chunk of the volume correction
constexpr int NRED = 8;            // partial sums per chunk (see reduce.cu)
constexpr int RING8 = 8;           // face entries per node kept at a fixed stride

// device status bits (Arrays::status[4 * d + 0])
constexpr int ST_NAN = 1;          // NaN / Inf in a node velocity or position
constexpr int ST_JUMP = 2;         // |qdot| > 1/2 in one step
constexpr int ST_SPREAD_OVF = 4;   // more than TILE_CAP nodes overlap a tile
constexpr int ST_COL_OVF = 8;      // more than MAXC crossings in a column
constexpr int ST_ESCAPE = 16;      // a node left the fluid in z
constexpr int ST_TIMEOUT = 32;     // a bounded wait for a bulk copy gave up
constexpr int ST_BAND_MISS = 64;   // a band tile lay outside the rows predicted for the step

// Per-droplet descriptor (device resident, read-only in kernels).
struct Drop {
    int nx, ny, nz, nzf, walls;
    int tx, ty, tz, ntiles;
    int64_t cell0, cells;          // first cell in the pooled (compact) cell arrays, count
    int64_t tile0;                 // first tile in the pooled tile arrays
    int64_t trow0;                 // first tile row (ty + tyc * tz) in the pooled tile-row arrays
    int64_t col0;                  // first column (nx*ny per droplet)
    int pitch;                     // population row pitch: nx rounded up to 16 elements
    int64_t pcell0, pcells;        // population planes: first padded cell, pitch*ny*nzf
    int64_t row0;                  // first row (y + ny z) in the pooled row arrays
    int node0, nnodes, tri0, ntri;
    int lb_block0, lb_nblocks;     // row groups of the stream-collide launch
    int lb_rows;                   // cell rows per group (consecutive y of one z-plane)
    int lb_gpp;                    // groups per z-plane: ceil(ny / lb_rows)
    int mass_block0, mass_nblocks; // blocks of the mass reduction
    int red_chunk0, red_nchunks;   // chunks of the mesh reductions
    float tau_out, tau_in, omega_out, omega_in;
    float rho0;
    float bf[3];                   // body force density
    float sigma, A, xi, hmin;
    float ks, ka;                  // Skalak moduli of an elastic membrane (0, 0: a droplet)
    int n, m, wetting, vartau, volcorr;
    double V0, R0;
    double inv_n, inv6V0;          // 1 / nnodes and 1 / (6 V0): the volume correction's fold multiplies
};

// Record written per node by the force kernel and read by the spread and
// the interpolation: base cell of the 4^3 support (fluid coordinates, x and
// y wrapped into the box), number of tiles the support touches (0: none in
// the fluid), kernel weights Psi along each axis for the support cells
// base-1 .. base+2, the nodal force phi_j and the node's droplet.
struct __align__(16) NodeRec {
    int bx, by, bz, key;
    float wx[4], wy[4], wz[4];
    float phi[3];
    int spare;
};
static_assert(sizeof(NodeRec) == 80, "the spread reads a record as five 16-byte words");

// Every device array of a context.  Lattice fields are pooled over droplets
// in the padded row layout of the populations: cell (x, row = y + ny z) of
// droplet d is index Drop::pcell0 + x + pitch * row; a 3-vector field stores
// component k at k * total_pcells + index.
struct Arrays {
    const Drop *drops;
    int ndrops;
    int pdl;                       // launch the kernels of the step with programmatic dependent launch
    int64_t total_cells;
    int64_t total_tiles;
    int total_nodes, total_tri;
    int lb_blocks_total;           // sum of Drop::lb_nblocks (row groups)
    int lb_stage_bytes;            // bytes of one shared-memory stage of the stream-collide kernel
    int64_t total_pcells;          // sum of Drop::pcells
    int64_t total_rows;            // sum of ny * nzf
    // lattice
    float *F;                      // 3 * total_pcells, force density: exactly 0 outside band tiles
    float4 *U;                     // total_pcells, velocity (ux, uy, uz, 0) per cell, interleaved so
                                   // that the interpolation reads a cell in one load (valid on band
                                   // rows only)
    uint32_t *tile_gen;            // tile is in the band of this step iff == *gen
    uint32_t *gen;                 // step generation counter (device)
    int *n_active;                 // 2: band tiles of this step / of the previous step
    int2 *active;                  // 2 * active_cap: band tiles, indexed by generation parity: the
                                   // pooled tile index and the tile's coordinates in its droplet
                                   // (tile_coords), so that readers need no divisions
    int active_cap;
    // per-tile node lists
    int *bin_cnt;                  // total_tiles: nodes listed in this step (returns to 0 in the spread)
    int *tile_list;                // TILE_CAP * total_tiles: node indices per tile, arrival order
    int *spread_done;              // blocks of the spread kernel finished (returns to 0)
    // stream-collide split: groups far from the membrane run concurrently
    // with the membrane kernels (see classify_groups in lb.cu)
    int64_t total_trows;           // sum of ty * tz (tile rows)
    uint32_t *rowgen;              // per tile row: last generation that put a tile of the row in the band
    uint8_t *candrow;              // per tile row: may hold band tiles in this step
    int *grp_list;                 // 2 * total_rows: groups near the band | groups far from it
    int *grp_cnt;                  // 2: their counts
    int *split_ok;                 // 1: the previous step's band predicts this step's (else all groups near)
    unsigned *bar_count;           // grid barrier of the cooperative kernels: arrivals
    unsigned *bar_flag;            // and release flag (flips at every barrier)
    // membrane
    double *qx, *qy, *qz;          // node positions (FP64) as advected; the volume correction of the
                                   // last step, when pending, is applied on reading (see red_out)
    double *px, *py, *pz;          // corrected positions of the step, written by the force kernel
    float4 *qh, *ql;               // q split into FP32 pairs (x, y, z, 0): qh = q rounded to FP32,
                                   // ql = q - qh rounded to FP32; written with q, read by the force
                                   // kernel for its relative vectors
    int *node_drop;                // droplet of each node
    const int *tri;                // 3 * total_tri global node indices
    const int *adj_start;          // total_nodes + 1
    const int *adj;                // (face << 2) | corner, faces in increasing order
    const int4 *ring;              // per entry of adj: the face's other corners (a, b), counter-
                                   // clockwise after the node, and (face << 2) | corner
    const int4 *ring8;             // RING8 entries per node: its first RING8 entries of ring, with
                                   // the node's face count in w (unused entries a = -1), so that
                                   // the force kernel needs no adj_start lookup first
    NodeRec *rec;                  // total_nodes
    // in/out
    int *col_cnt;                  // crossings per column
    double *col_z;                 // MAXC crossings per column (sorted)
    int64_t total_cols;
    int *face_drop;                // droplet of each face
    const float4 *fref;            // per face, from the mesh given at set-up: S = H^-1 of the
                                   // reference edge Gram matrix H (x = S11, y = S12, z = S22)
                                   // and the reference area A0 (w); null when no droplet is elastic
    // reductions
    double *red_part;              // NRED * chunks (volume-correction partials)
    double *red_out;               // NRED * ndrops: k = (V0/V)^(1/3), cx, cy, cz, V, pending (1: the
                                   // positions q are to be read as c + (q - c) k), -, -
    int *vc_done;                  // per droplet: finished chunks (returns to 0)
    double *mass_part;
    int *status;                   // 4 ints per droplet: flags (ST_*), -, -, -
    uint8_t *clamped;              // per node: 1 if the near-wall guard clamped it in this step
};

// Tracing (iblb_trace_step): once its wait on the previous kernel returned,
// every warp of the step's kernels writes %globaltimer (ns) into
// trace[k * TRACE_WARPS + w] for kernel k (TraceKernel) and warp w of the
// launch (blockIdx.x * warps per block + warp; warps from TRACE_WARPS on are
// not recorded).  A kernel's end is read as the next kernel's first start
// (TR_END: a marker kernel launched after the step), which programmatic
// dependent launch places after its last exit.  The stamps live in separate
// instantiations of the kernels (template flag TR, the buffer as a trailing
// argument), launched only while a host-side buffer is set: the untraced
// kernels carry no stamp code (a run-time check, an exit stamp or a kernel
// parameter read each cost measurable time in the chained step).
enum TraceKernel { TR_FORCE = 0, TR_SPREAD = 1, TR_LB = 2, TR_INTERP = 3, TR_VC = 4, TR_END = 5, TRACE_KERNELS = 5 };
constexpr int TRACE_WARPS = 32768;
__device__ __forceinline__ void trace_start(unsigned long long *trace, int k)
{
    if (trace == nullptr || (threadIdx.x & 31) != 0)
        return;
    const unsigned w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= (unsigned)TRACE_WARPS)
        return;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    trace[(size_t)k * TRACE_WARPS + w] = t;
}
// Launch the traced instantiations with this stamp buffer from now on
// (nullptr: the plain ones); host-side state of the membrane launches and of
// the stream-collide launches.
void set_trace_ib(unsigned long long *trace);
void set_trace_lb(unsigned long long *trace);
// The step's trailing marker (one warp): its start ends the last kernel.
cudaError_t launch_trace_marker(const Arrays &a, unsigned long long *trace, cudaStream_t s);

// Programmatic dependent launch: a kernel of the step may be launched while
// the previous one finishes; griddep_wait() returns once the previous kernel
// has completed and its writes are visible, and it is the first statement of
// every kernel of the step (a no-op for a kernel launched without the
// attribute).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with or without programmatic dependent launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                     Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// tile coordinates (tx < 2048, ty < 2048, tz < 1024) packed in one int
__host__ __device__ inline int tile_coords(int tx, int ty, int tz) { return tx | (ty << 11) | (tz << 22); }

__host__ __device__ inline int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// floor(a / b) for b > 0
__host__ __device__ inline int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Host-side launchers (lb.cu, ib.cu, inout.cu, reduce.cu, fields.cu).
struct LaunchCfg {
    int lb_blocks_per_sm;          // resident stream-collide blocks per SM (0: as many as fit)
    int lb_row_mult;               // cell rows per group = lb_row_mult * lb_rows_per_group(nx)
    int sm_count;
    int lb_stages;                 // shared-memory stages of the stream-collide pipeline (2..8)
    int ib_blocks_per_sm;          // blocks per SM of the cooperative membrane kernels (0: all that fit)
    int lb_group_cells = 0;        // if > 0: about this many cells per group (whole rows), in place of the multiplier
};
int lb_rows_per_group(int nx);     // 256-thread groups: max(1, 256 / nx) rows
// bytes of one stage of the stream-collide kernel: 19 population rows and 3
// force rows per cell row and the band flag (128-byte multiple)
int lb_stage_bytes(int rows, int pitch, int storage_bytes);

// Stream-collide over every group (list == nullptr) or over the groups
// list[0 .. *count); no_force: the groups carry no force (skip the band test).
cudaError_t launch_lb(const Arrays &a, int storage, const void *src, void *dst, bool vartau,
                      const LaunchCfg &cfg, cudaStream_t s, const int *list = nullptr, const int *count = nullptr,
                      bool no_force = false, int blocks_per_sm = -1);
// Split the stream-collide groups of the coming step into those whose rows
// may meet its band (within one tile row of the previous step's band) and
// the others; also marks the tile rows that may hold band tiles.
cudaError_t launch_classify(const Arrays &a, cudaStream_t s);
cudaError_t launch_node_force(const Arrays &a, cudaStream_t s);
cudaError_t launch_spread(const Arrays &a, cudaStream_t s);
cudaError_t launch_inout(const Arrays &a, cudaStream_t s);
cudaError_t launch_interp_advect(const Arrays &a, cudaStream_t s);
// cooperative kernels: forces + tile lists + spread; advection + volume correction
// (per_sm: resident blocks per SM of the cooperative grid, 0 = as many as fit)
cudaError_t launch_ib_front(const Arrays &a, int per_sm, cudaStream_t s);
cudaError_t launch_ib_back(const Arrays &a, int n_chunks_total, bool volcorr, int per_sm, cudaStream_t s);
// FP64 volume and centroid of every droplet with volume correction and the
// rescale of its nodes (one cooperative launch)
cudaError_t launch_volume_correction(const Arrays &a, int n_chunks_total, cudaStream_t s);
cudaError_t launch_mass(const Arrays &a, int storage, const void *f, double *d_out, int mass_blocks,
                        cudaStream_t s);
// Corrected positions of every node into a.px, a.py, a.pz (the pending
// volume correction applied; a plain copy where none is pending).
cudaError_t launch_corrected_positions(const Arrays &a, cudaStream_t s, double *xyz = nullptr, int node0 = 0,
                                       int n = 0);
// Droplet k's nodes node0 .. node0 + n - 1 set from the device array xyz
// (x, y, z per node), with no volume correction pending for the droplet.
cudaError_t launch_set_nodes(const Arrays &a, const double *xyz, int node0, int n, int k, cudaStream_t s);
// Observables of one mesh: node j at q*[j * stride]; tri holds node indices
// into q*; nodes node0 .. node0 + nnodes - 1.  Writes 13 doubles to h_out
// (volume, area, centroid[3], zmin, zmax, theta_R0, theta_RV, rc_cut,
// rc_flat, n_cut, chi_flat) and synchronises s.
int64_t observe_scratch_doubles(int n_nodes, int n_tri);
cudaError_t launch_observe_view(const double *qx, const double *qy, const double *qz, int stride,
                                const int *tri, int ntri, int node0, int nnodes, double R0, double zcut_frac,
                                double eps_flat, double *scratch, double *h_out, cudaStream_t s);
// The same for a context's droplet (positions with stride 1, and the
// near-wall guard's per-node flags, counted as a fourteenth value) without
// the synchronisation: the kernels and a copy of 32 raw doubles to hv (host,
// pinned) are enqueued on s; once s has passed them, finish_observe turns hv
// into the 14 values.
cudaError_t enqueue_observe(const double *qx, const double *qy, const double *qz, const uint8_t *clamped,
                            const int *tri, int ntri, int node0, int nnodes, double R0, double zcut_frac,
                            double eps_flat, double *scratch, double *hv, cudaStream_t s);
void finish_observe(const double *hv, double R0, double *h_out);
// Bring the code of the observation kernels onto the current device now
// (module loading is lazy by default, and a load allocates device memory).
cudaError_t preload_observe_kernels();

// Conversions of droplet d (device pointers; `cells` = that droplet's cells).
cudaError_t launch_export_populations(const Arrays &a, int d, int storage, const void *f, double *out,
                                      int64_t cells, cudaStream_t s);
cudaError_t launch_import_populations(const Arrays &a, int d, int storage, void *f, const double *in,
                                      int64_t cells, cudaStream_t s);
cudaError_t launch_export_macros(const Arrays &a, int d, int storage, const void *f, double *rho, double *u,
                                 int64_t cells, cudaStream_t s);
cudaError_t launch_export_force(const Arrays &a, int d, double *F, int64_t cells, cudaStream_t s);
cudaError_t launch_export_inside(const Arrays &a, int d, uint8_t *inside, int64_t cells, cudaStream_t s);
cudaError_t launch_init_populations(const Arrays &a, int storage, void *f, cudaStream_t s);

}  // namespace iblb
