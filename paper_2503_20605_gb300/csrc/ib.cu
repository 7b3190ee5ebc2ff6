// ib.cu -- the membrane side of the IB-LB step:
//   * nodal forces: surface tension phi_sigma,j = -sigma dA/dq_j (Sec. II B)
//     plus the wall interaction phi_Pi,j = -(chi_j/3) Pi(h_j) n_j (Sec. II C);
//     four lanes per node share its incident faces, partial sums meet in a
//     fixed shuffle tree, one lane per axis takes the kernel support;
//     every node is listed in the 4^3 tiles its 4x4x4 kernel support touches
//     (at most 8, or 27 across a partial periodic tile), and the tiles with a
//     node form the band;
//   * force spreading F(x) = sum_j phi_j Delta(q_j - x) (eq. force_spread) as
//     a deterministic gather: every band tile orders its nodes by index and
//     each cell adds their contributions in that order, so the result depends
//     neither on launch shapes nor on the other droplets of a batch;
//   * interpolation qdot_j = sum_x U(x) Delta(q_j - x) (eq. vel_interpolation)
//     and forward-Euler advection q_j += qdot_j, 16 lanes per node;
//   * the volume correction q <- c + (q - c)(V0/V)^(1/3) about the node
//     centroid (not in the paper), FP64 volume and centroid per droplet.
// The work runs either as separate kernels or as two cooperative kernels
// (forces + lists + spread before the stream-collide kernel; advection +
// volume correction after it) whose phases are separated by a grid barrier:
// the same device functions, the same arithmetic, bit-identical results.
// Node positions are FP64 so that edge vectors and kernel offsets are exact
// before they are rounded to FP32 for the force and kernel arithmetic.
// This file is compiled without implicit fused multiply-adds (-fmad=false):
// its device functions are inlined into both the separate and the
// cooperative kernels, and only the explicit fmaf calls fuse, so that both
// give the same bits.
#include <algorithm>

#include <cuda/atomic>

#include "iblb_internal.h"
#include "reduce_util.cuh"

namespace iblb {

namespace {

unsigned long long *g_trace_ib = nullptr;   // host: stamp buffer of a traced step (see iblb_trace_step)

constexpr int IB_THREADS = 128;  // block size of the other membrane kernels (256 measured 0.3 us slower)
constexpr int SPREAD_PARTS = 4;  // parts of a tile's sorted node list, summed separately per cell
constexpr int SP_THREADS = 128;  // block size of the separate spread kernel and its blocks per SM: 1216
constexpr int SP_PER_SM = 8;     // blocks, so that a droplet's band (about 1200 tiles at R = 24) takes
                                 // one round (256-thread blocks, four per SM, took two: 2.6 us more)
constexpr int SPREAD_STAGE = 256;  // records of a tile staged in shared memory at a time
constexpr int VC_RB = VC_ITEMS;  // threads per volume-correction chunk
constexpr long long BARRIER_CYCLES = 4000000000LL;      // ~2 s: bounded grid-barrier wait

__device__ __forceinline__ float ipow(float r, int k)
{
    float p = 1.0f;
    for (int i = 0; i < k; ++i)
        p *= r;
    return p;
}

__device__ __forceinline__ int find_drop_tile(const Drop *D, int n, int64_t t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].tile0 <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The volume correction of a step (not in the paper) is kept pending: the
// stored positions q are those after advection, and the correction
// q' = c + (q - c) k computed from them is applied wherever positions are
// read, until the next advection replaces q.  Every reader applies it with
// the same three individually rounded FP64 operations, so a position reads
// the same wherever it is read.
struct Corr {
    bool on;
    double k, cx, cy, cz;
};
__device__ __forceinline__ Corr load_corr(const Arrays &a, int d)
{
    const double *r = a.red_out + (int64_t)NRED * d;
    Corr c;
    c.on = r[5] != 0.0;
    c.k = r[0];
    c.cx = r[1];
    c.cy = r[2];
    c.cz = r[3];
    return c;
}
__device__ __forceinline__ double corr1(double q, double c, double k)
{
    return __dadd_rn(c, __dmul_rn(__dsub_rn(q, c), k));
}

// x rounded to nearest (ties to even) FP32 by integer operations on its
// bits: equal to the FP64 -> FP32 conversion for |x| in FP32's normal range,
// zero, infinities and NaN; smaller magnitudes give a signed zero.  The
// conversion instruction costs about as much issue as two FP64 additions on
// this GPU, the integer operations a small fraction of one.
__device__ __forceinline__ float dtof_rn(double x)
{
    const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
    const unsigned s = h & 0x80000000u;
    const int e = (int)((h >> 20) & 0x7ffu) - 896;          // FP32 biased exponent
    const unsigned m = ((h & 0xfffffu) << 3) | (l >> 29);    // the top 23 fraction bits
    const unsigned r = l & 0x1fffffffu;                      // the 29 bits below them
    unsigned b = ((unsigned)e << 23) + m;
    b += (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u;   // a carry moves into the exponent
    if (e <= 0)
        b = 0u;
    if (e >= 255)
        b = ((h & 0x7ff00000u) == 0x7ff00000u && ((h & 0xfffffu) | l)) ? 0x7fc00000u : 0x7f800000u;
    return __uint_as_float(s | b);
}

// One coordinate of q_a - q_j from the FP32 pairs of the two positions: the
// hi parts of nearby positions differ exactly, the lo parts carry the rest.
__device__ __forceinline__ float rel_coord(float ah, float al, float jh, float jl)
{
    return __fadd_rn(__fsub_rn(ah, jh), __fsub_rn(al, jl));
}

// One incident face (j, a, b) of a node: relative corner vectors r_a, r_b
// (already dilated by a pending volume correction), accumulated into the
// node's area gradient g, normal sum n, area sum chi and elastic force e.
template <bool EL>
__device__ __forceinline__ void face_terms(const Arrays &a, int4 en, float rax, float ray, float raz, float rbx,
                                           float rby, float rbz, bool elastic, float ks3, float ka3, float &gx,
                                           float &gy, float &gz, float &nx, float &ny, float &nz, float &chi,
                                           float &ex, float &ey, float &ez)
{
    const float Nx = ray * rbz - raz * rby;
    const float Ny = raz * rbx - rax * rbz;
    const float Nz = rax * rby - ray * rbx;
    const float len = sqrtf(Nx * Nx + Ny * Ny + Nz * Nz);
    const float il = 1.0f / len;
    const float hx = Nx * il, hy = Ny * il, hz = Nz * il;
    // dA/dq_j = 1/2 n x (q_prev - q_next), (prev, j, next) = (b, j, a)
    const float dx = rbx - rax, dy = rby - ray, dz = rbz - raz;
    const float ax = 0.5f * (hy * dz - hz * dy), ay = 0.5f * (hz * dx - hx * dz), az = 0.5f * (hx * dy - hy * dx);
    gx += ax;
    gy += ay;
    gz += az;
    if (EL && elastic) {
        // Skalak energy against the reference triangle (Sec. II B's
        // framework): with S = H^-1 and A0 from the reference,
        // b = (S11 e1.e1 + 2 S12 e1.e2 + S22 e2.e2) / 2 - 1, r = A / A0,
        // phi_k = -(A0 w_a / A) dA/dq_k - A0 w_b (1/2) dtr/dq_k, with the
        // face's edges e1 = q1 - q0, e2 = q2 - q0 in its own corner order
        // (j is corner k: (j, a, b) rotated)
        const int t = en.z >> 2, k = en.z & 3;
        float e1x, e1y, e1z, e2x, e2y, e2z;
        if (k == 0) {
            e1x = rax; e1y = ray; e1z = raz;
            e2x = rbx; e2y = rby; e2z = rbz;
        } else if (k == 1) {
            e1x = -rbx; e1y = -rby; e1z = -rbz;
            e2x = rax - rbx; e2y = ray - rby; e2z = raz - rbz;
        } else {
            e1x = rbx - rax; e1y = rby - ray; e1z = rbz - raz;
            e2x = -rax; e2y = -ray; e2z = -raz;
        }
        const float4 R = a.fref[t];
        const float g11 = e1x * e1x + e1y * e1y + e1z * e1z, g12 = e1x * e2x + e1y * e2y + e1z * e2z;
        const float g22 = e2x * e2x + e2y * e2y + e2z * e2z;
        const float b = 0.5f * (R.x * g11 + 2.0f * R.y * g12 + R.z * g22) - 1.0f;
        const float r = 0.5f * len / R.w;
        const float cA = r * (ka3 * (r * r - 1.0f) - ks3), cB = R.w * ks3 * (2.0f * b + 1.0f);
        const float h1x = R.x * e1x + R.y * e2x, h1y = R.x * e1y + R.y * e2y, h1z = R.x * e1z + R.y * e2z;
        const float h2x = R.y * e1x + R.z * e2x, h2y = R.y * e1y + R.z * e2y, h2z = R.y * e1z + R.z * e2z;
        const float tx = k == 0 ? -(h1x + h2x) : (k == 1 ? h1x : h2x);
        const float ty = k == 0 ? -(h1y + h2y) : (k == 1 ? h1y : h2y);
        const float tz = k == 0 ? -(h1z + h2z) : (k == 1 ? h1z : h2z);
        ex -= cA * ax + cB * tx;
        ey -= cA * ay + cB * ty;
        ez -= cA * az + cB * tz;
    }
    nx += hx;
    ny += hy;
    nz += hz;
    chi += 0.5f * len;
}

// The four weights of the 4-point kernel at the support cells base-1 ..
// base+2 of one axis, for the node's offset f in [0, 1) from the base: with
// s = sqrt(1/4 + f - f^2), Psi(1 + f) = 3/8 - f/4 - s/4, Psi(f) = 3/8 - f/4
// + s/4, Psi(1 - f) = 1/8 + f/4 + s/4 and Psi(2 - f) = 1/8 + f/4 - s/4 (both
// branches of Psi, Sec. II A, evaluated at these four distances share s).
__device__ __forceinline__ void psi4(float f, float *w)
{
    const float s = 0.25f * sqrtf(0.25f + f - f * f);
    const float p = 0.375f - 0.25f * f, q = 0.125f + 0.25f * f;
    w[0] = p - s;
    w[1] = p + s;
    w[2] = q + s;
    w[3] = q - s;
}

// The distinct tiles (in increasing cell order) holding the support cells
// b-1 .. b+2 of one axis of n cells: wrapped on a periodic axis, clipped to
// [0, n) otherwise; at most 3 (a partial last tile of a periodic axis).
__device__ __forceinline__ int support_tiles3(int b, int n, bool periodic, int &t0, int &t1, int &t2)
{
    int cnt = 0;
    t0 = t1 = t2 = -1;
#pragma unroll
    for (int k = -1; k <= 2; ++k) {
        int c = b + k;
        if (periodic)
            c = wrapi(c, n);
        else if (c < 0 || c >= n)
            continue;
        const int t = c >> 2;
        if (t == t0 || t == t1 || t == t2)
            continue;
        if (cnt == 0)
            t0 = t;
        else if (cnt == 1)
            t1 = t;
        else
            t2 = t;
        ++cnt;
    }
    return cnt;
}

// Forces of node j, NL = 4 lanes per node.  The node's incident faces are
// listed as (a, b, t << 2 | k): the face's other two corners in
// counter-clockwise order about the outward normal -- the face is (j, a, b)
// -- and the face and the corner j takes in it.  Lane l takes the faces l,
// l + 4, ...; with r_a = q_a - q_j and r_b = q_b - q_j (from the FP32 pairs
// of the positions, dilated by k when a volume correction is pending) a
// face's normal is r_a x r_b, its area half its length, and dA/dq_j =
// 1/2 n x (r_b - r_a).  The lanes' sums meet in a fixed shuffle tree.  Lane
// c < 3 takes axis c of the node (its corrected coordinate, kernel support
// and weights) and lane 3 the nodal force; the node is listed in the 4^3
// tiles its kernel support touches, the lanes sharing the tiles: its slot in
// a tile's list (TILE_CAP slots per tile) comes from the tile's counter, and
// the node that takes slot 0 stamps the tile with the step's generation gen
// and appends it to the band list.  The axis work and the listing depend on
// the node's own position only: they run while the first faces'
// neighbour positions are in flight.  Every lane of the warp takes part
// (the shuffles span whole quads).
constexpr int NL = 4;
template <bool EL>     // EL: some droplet of the launch has an elastic membrane (a.fref set)
__device__ __forceinline__ void node_forces(const Arrays &a, int64_t gid, uint32_t gen)
{
    const int j = (int)(gid >> 2), l = (int)(gid & 3);
    const bool valid = j < a.total_nodes;
    float gx = 0.f, gy = 0.f, gz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f, chi = 0.f;
    float ex = 0.f, ey = 0.f, ez = 0.f;     // elastic (Skalak) force, when the droplet has moduli
    int d = 0;
    Corr cr = {false, 1.0, 0.0, 0.0, 0.0};
    double qx0 = 0.0, qy0 = 0.0, qz0 = 0.0;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 jh = zero4, jl = zero4;
    // the node's first RING8 faces at a fixed stride (lane l: entries l and
    // l + 4, the first pass), further ones (a face count above RING8) from
    // the list; the first pass's neighbour positions are loaded at once
    int4 f0 = make_int4(-1, -1, 0, 0), f1 = f0;
    int nfaces = 0;
    float4 a0h = zero4, a0l = zero4, b0h = zero4, b0l = zero4, a1h = zero4, a1l = zero4, b1h = zero4, b1l = zero4;
    if (valid) {
        d = a.ndrops == 1 ? 0 : a.node_drop[j];   // (one droplet: no lookup on the critical path)
        cr = load_corr(a, d);
        qx0 = a.qx[j];
        qy0 = a.qy[j];
        qz0 = a.qz[j];
        jh = a.qh[j];
        jl = a.ql[j];
        f0 = a.ring8[(int64_t)RING8 * j + l];
        f1 = a.ring8[(int64_t)RING8 * j + l + NL];
        nfaces = f0.w;
        if (l < nfaces) {
            a0h = a.qh[f0.x];
            a0l = a.ql[f0.x];
            b0h = a.qh[f0.y];
            b0l = a.ql[f0.y];
        }
        if (l + NL < nfaces) {
            a1h = a.qh[f1.x];
            a1l = a.ql[f1.x];
            b1h = a.qh[f1.y];
            b1l = a.ql[f1.y];
        }
    }
    // axis c = l of the node (lanes 0 .. 2): corrected coordinate, kernel
    // support and weights
    const Drop &D = a.drops[d];
    const int ax = l < 3 ? l : 2;
    double q = ax == 0 ? qx0 : (ax == 1 ? qy0 : qz0);
    if (cr.on)
        q = corr1(q, ax == 0 ? cr.cx : (ax == 1 ? cr.cy : cr.cz), cr.k);
    const int qb = threadIdx.x & 28;      // the quad's first lane
    const int sane_l = fabs(q) < 1e8 ? 1 : 0;
    const bool sane = __shfl_sync(0xffffffffu, sane_l, qb | 0) && __shfl_sync(0xffffffffu, sane_l, qb | 1) &&
                      __shfl_sync(0xffffffffu, sane_l, qb | 2);
    int b = 0, nt = 0, t0 = -1, t1 = -1, t2 = -1;
    float w[4] = {0.f, 0.f, 0.f, 0.f};
    if (valid && l < 3 && sane) {
        const double fb = floor(q);
        const float f = dtof_rn(q - fb);
        const int n = ax == 0 ? D.nx : (ax == 1 ? D.ny : D.nzf);
        if (ax < 2) {
            b = wrapi((int)fb % n, n);
            nt = support_tiles3(b, n, true, t0, t1, t2);
        } else {
            b = (int)fb - D.walls;
            if (!D.walls)
                b = wrapi(b % D.nz, D.nz);
            nt = support_tiles3(b, n, !D.walls, t0, t1, t2);
        }
        psi4(f, w);
    }
    // the z coordinate (lane 2) for the wall interaction; the tile counts
    // and tiles of every axis for the listing
    const double qz = __shfl_sync(0xffffffffu, q, qb | 2);
    const int ntx = __shfl_sync(0xffffffffu, nt, qb | 0), nty = __shfl_sync(0xffffffffu, nt, qb | 1),
              ntz = __shfl_sync(0xffffffffu, nt, qb | 2);
    const int tx0 = __shfl_sync(0xffffffffu, t0, qb | 0), tx1 = __shfl_sync(0xffffffffu, t1, qb | 0),
              tx2 = __shfl_sync(0xffffffffu, t2, qb | 0);
    const int ty0 = __shfl_sync(0xffffffffu, t0, qb | 1), ty1 = __shfl_sync(0xffffffffu, t1, qb | 1),
              ty2 = __shfl_sync(0xffffffffu, t2, qb | 1);
    const int tz0 = __shfl_sync(0xffffffffu, t0, qb | 2), tz1 = __shfl_sync(0xffffffffu, t1, qb | 2),
              tz2 = __shfl_sync(0xffffffffu, t2, qb | 2);
    const int ncombo = ntx * nty * ntz;
    NodeRec &rec = a.rec[valid ? j : 0];
    if (valid && l < 3) {
        // the corrected coordinate, for the in/out test and the advection of this step
        (ax == 0 ? a.px : (ax == 1 ? a.py : a.pz))[j] = q;
        (&rec.bx)[ax] = b;
        float *rw = ax == 0 ? rec.wx : (ax == 1 ? rec.wy : rec.wz);
        *reinterpret_cast<float4 *>(rw) = make_float4(w[0], w[1], w[2], w[3]);
    }
    // the node's tiles, shared by the four lanes: every counter's atomic is
    // issued before any result is used (a support across a partial periodic
    // tile can touch up to 27 tiles)
    const int cur = (int)(gen & 1u);
    for (int c0 = l; valid && c0 < ncombo; c0 += 2 * NL) {
        int64_t tl[2], trw[2];
        int rk[2], tc[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = c0 + i * NL;
            if (c < ncombo) {
                const int ix = c % ntx, iy = (c / ntx) % nty, iz = c / (ntx * nty);
                const int tx = ix == 0 ? tx0 : (ix == 1 ? tx1 : tx2);
                const int ty = iy == 0 ? ty0 : (iy == 1 ? ty1 : ty2);
                const int tz = iz == 0 ? tz0 : (iz == 1 ? tz1 : tz2);
                tl[i] = D.tile0 + tx + (int64_t)D.tx * (ty + (int64_t)D.ty * tz);
                trw[i] = D.trow0 + ty + (int64_t)D.ty * tz;
                tc[i] = tile_coords(tx, ty, tz);
                rk[i] = atomicAdd(&a.bin_cnt[tl[i]], 1);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            if (c0 + i * NL >= ncombo)
                continue;
            const int64_t t = tl[i];
            const int rank = rk[i];
            if (rank == 0) {        // first node of the tile: the tile joins the band
                a.tile_gen[t] = gen;
                const int slot = atomicAdd(&a.n_active[cur], 1);
                if (slot < a.active_cap)
                    a.active[(int64_t)cur * a.active_cap + slot] = make_int2((int)t, tc[i]);
                // its tile row too; the stream-collide rows run before this
                // step's band was known assumed that this row could not hold
                // band tiles
                a.rowgen[trw[i]] = gen;
                if (a.grp_cnt[2] && !a.candrow[trw[i]])
                    atomicOr(&a.status[4 * d], ST_BAND_MISS);
            }
            if (rank < TILE_CAP)
                a.tile_list[t * TILE_CAP + rank] = j;
            else
                atomicOr(&a.status[4 * d], ST_SPREAD_OVF);
        }
    }
    // the faces: the first pass from the positions loaded above, then any
    // further passes (nodes with more than RING8 faces)
    if (valid) {
        const float kf = cr.on ? dtof_rn(cr.k) : 1.0f;
        float ks3 = 0.0f, ka3 = 0.0f;
        if (EL) {
            ks3 = a.drops[d].ks * (1.0f / 3.0f);
            ka3 = a.drops[d].ka * (1.0f / 3.0f);
        }
        const bool elastic = EL && (ks3 != 0.0f || ka3 != 0.0f);
        if (l < nfaces)
            face_terms<EL>(a, f0, rel_coord(a0h.x, a0l.x, jh.x, jl.x) * kf, rel_coord(a0h.y, a0l.y, jh.y, jl.y) * kf,
                           rel_coord(a0h.z, a0l.z, jh.z, jl.z) * kf, rel_coord(b0h.x, b0l.x, jh.x, jl.x) * kf,
                           rel_coord(b0h.y, b0l.y, jh.y, jl.y) * kf, rel_coord(b0h.z, b0l.z, jh.z, jl.z) * kf,
                           elastic, ks3, ka3, gx, gy, gz, nx, ny, nz, chi, ex, ey, ez);
        if (l + NL < nfaces)
            face_terms<EL>(a, f1, rel_coord(a1h.x, a1l.x, jh.x, jl.x) * kf, rel_coord(a1h.y, a1l.y, jh.y, jl.y) * kf,
                           rel_coord(a1h.z, a1l.z, jh.z, jl.z) * kf, rel_coord(b1h.x, b1l.x, jh.x, jl.x) * kf,
                           rel_coord(b1h.y, b1l.y, jh.y, jl.y) * kf, rel_coord(b1h.z, b1l.z, jh.z, jl.z) * kf,
                           elastic, ks3, ka3, gx, gy, gz, nx, ny, nz, chi, ex, ey, ez);
        const int e0 = nfaces > RING8 ? a.adj_start[j] : 0;
        for (int eb = l + 2 * NL; eb < nfaces; eb += 2 * NL) {
            // two faces per pass, every load issued before the arithmetic
            const bool two = eb + NL < nfaces;
            const int4 en0 = a.ring[e0 + eb];
            const int4 en1 = two ? a.ring[e0 + eb + NL] : en0;
            const float4 c0h = a.qh[en0.x], c0l = a.ql[en0.x], d0h = a.qh[en0.y], d0l = a.ql[en0.y];
            const float4 c1h = a.qh[en1.x], c1l = a.ql[en1.x], d1h = a.qh[en1.y], d1l = a.ql[en1.y];
            face_terms<EL>(a, en0, rel_coord(c0h.x, c0l.x, jh.x, jl.x) * kf, rel_coord(c0h.y, c0l.y, jh.y, jl.y) * kf,
                           rel_coord(c0h.z, c0l.z, jh.z, jl.z) * kf, rel_coord(d0h.x, d0l.x, jh.x, jl.x) * kf,
                           rel_coord(d0h.y, d0l.y, jh.y, jl.y) * kf, rel_coord(d0h.z, d0l.z, jh.z, jl.z) * kf,
                           elastic, ks3, ka3, gx, gy, gz, nx, ny, nz, chi, ex, ey, ez);
            if (two)
                face_terms<EL>(a, en1, rel_coord(c1h.x, c1l.x, jh.x, jl.x) * kf,
                               rel_coord(c1h.y, c1l.y, jh.y, jl.y) * kf, rel_coord(c1h.z, c1l.z, jh.z, jl.z) * kf,
                               rel_coord(d1h.x, d1l.x, jh.x, jl.x) * kf, rel_coord(d1h.y, d1l.y, jh.y, jl.y) * kf,
                               rel_coord(d1h.z, d1l.z, jh.z, jl.z) * kf, elastic, ks3, ka3, gx, gy, gz, nx, ny, nz,
                               chi, ex, ey, ez);
        }
    }
    for (int o = NL / 2; o >= 1; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
        nx += __shfl_xor_sync(0xffffffffu, nx, o);
        ny += __shfl_xor_sync(0xffffffffu, ny, o);
        nz += __shfl_xor_sync(0xffffffffu, nz, o);
        chi += __shfl_xor_sync(0xffffffffu, chi, o);
    }
    if (EL)
        for (int o = NL / 2; o >= 1; o >>= 1) {
            ex += __shfl_xor_sync(0xffffffffu, ex, o);
            ey += __shfl_xor_sync(0xffffffffu, ey, o);
            ez += __shfl_xor_sync(0xffffffffu, ez, o);
        }
    if (valid && l == 3) {
        rec.key = ncombo;
        rec.spare = d;
        uint8_t clamped = 0;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (!sane) {
            atomicOr(&a.status[4 * d], ST_NAN);
        } else {
            px = -D.sigma * gx;
            py = -D.sigma * gy;
            pz = -D.sigma * gz;
            if (EL) {
                px += ex;
                py += ey;
                pz += ez;
            }
            if (D.wetting) {
                float h = dtof_rn(qz - 0.5);
                if (h < D.hmin) {
                    h = D.hmin;
                    clamped = 1;
                }
                const float r0 = D.xi / h;
                const float Pi = D.A * (ipow(r0, D.n) - ipow(r0, D.m));
                const float inl = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
                const float sc = -(chi * (1.0f / 3.0f)) * Pi * inl;
                px += sc * nx;
                py += sc * ny;
                pz += sc * nz;
            }
            if (ncombo == 0)
                atomicOr(&a.status[4 * d], ST_ESCAPE);
        }
        rec.phi[0] = px;
        rec.phi[1] = py;
        rec.phi[2] = pz;
        a.clamped[j] = clamped;
    }
}

// offset of cell X from support base b on a periodic axis of n cells,
// mapped into the support window [-1, 2] when it lies there
__device__ __forceinline__ int per_off(int X, int b, int n)
{
    int d = X - b;
    if (d < -1)
        d += n;
    else if (d > 2)
        d -= n;
    return d;
}

// Shared memory of one spread block: the keys (node indices) of a tile's
// nodes in arrival order and, for a window of SPREAD_STAGE consecutive ranks
// of the keys in increasing order, one 16-float record per node: its kernel
// weights at the tile's four cells of each axis, x at 0..3, y at 4..7, z at
// 8..11 (0 where the cell lies outside the node's support), and its force at
// 12..14.
struct SpreadSmem {
    __align__(16) int node[TILE_CAP];
    __align__(16) float rec[SPREAD_STAGE][16];
    __align__(16) float part[3][SPREAD_PARTS][TILE_CELLS];
    int last;
};

// Kernel weights of one axis at the four cells T0 .. T0+3 of a tile: w[d+1]
// where the cell is at offset d in -1 .. 2 from the support base b (wrapped
// on a periodic axis of n cells), else 0.
__device__ __forceinline__ void tile_weights(int T0, int b, int n, bool periodic, const float *w, float *out)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int d = periodic ? per_off(T0 + c, b, n) : T0 + c - b;
        out[c] = (d >= -1 && d <= 2) ? w[d + 1] : 0.0f;
    }
}

// Tiles of the previous band that are not in this step's band: zero their
// force so that F vanishes outside the band (band tiles are rewritten).
// Block bid of nb (NT threads) takes NT / 64 tiles per pass, 64 threads each.
// The first tile of a thread's pass is looked up by zero_left_first (its
// loads can be issued when the kernel starts) and zeroed at the end with the
// others: the spread writes only tiles of this step's band, so the order
// does not matter.
struct LeftTile {
    int64_t T = -1;
    int coords = 0;
    uint32_t g = 0;
};
template <int NT>
__device__ __forceinline__ LeftTile zero_left_first(const Arrays &a, int cur, int bid)
{
    constexpr int TPB = NT / TILE_CELLS;
    LeftTile lt;
    const int it = bid * TPB + threadIdx.x / TILE_CELLS;
    if (it < min(a.n_active[cur ^ 1], a.active_cap)) {
        const int2 e = a.active[(int64_t)(cur ^ 1) * a.active_cap + it];
        lt.T = e.x;
        lt.coords = e.y;
        lt.g = a.tile_gen[lt.T];
    }
    return lt;
}

template <int NT>
__device__ void zero_left_tiles(const Arrays &a, uint32_t gen, int cur, int bid, int nb, LeftTile first)
{
    constexpr int TPB = NT / TILE_CELLS;
    const int tid = threadIdx.x;
    const int nprev = min(a.n_active[cur ^ 1], a.active_cap);
    const int2 *plist = a.active + (int64_t)(cur ^ 1) * a.active_cap;
    for (int it = bid * TPB + tid / TILE_CELLS; it < nprev; it += nb * TPB) {
        const bool pre = it == bid * TPB + tid / TILE_CELLS && first.T >= 0;
        const int2 e = pre ? make_int2((int)first.T, first.coords) : plist[it];
        const int64_t T = e.x;
        if ((pre ? first.g : a.tile_gen[T]) == gen)
            continue;
        const int d = a.ndrops == 1 ? 0 : find_drop_tile(a.drops, a.ndrops, T);
        const Drop &D = a.drops[d];
        const int cell = tid & (TILE_CELLS - 1);
        const int X = 4 * (e.y & 2047) + (cell & 3);
        const int Y = 4 * ((e.y >> 11) & 2047) + ((cell >> 2) & 3);
        const int Z = 4 * (e.y >> 22) + (cell >> 4);
        if (X < D.nx && Y < D.ny && Z < D.nzf) {
            const int64_t g = D.pcell0 + X + (int64_t)D.pitch * (Y + (int64_t)D.ny * Z);
            a.F[g] = 0.0f;
            a.F[a.total_pcells + g] = 0.0f;
            a.F[2 * a.total_pcells + g] = 0.0f;
        }
    }
}

// Band tiles bid, bid + nb, ...: the tile's node indices are staged and
// ranked (rank = how many of the tile's nodes have a smaller index); the
// records of ranks w0 .. w0 + SPREAD_STAGE - 1 are placed in shared memory
// in rank order, one window after the other.  Every cell adds SPREAD_PARTS
// consecutive parts of the sorted list separately (a thread per part and
// x-row of four cells, its sums carried from window to window) and the parts
// are summed in a fixed order, so every cell's force is the same for any
// launch shape, block size and window size.  The tile's counter returns to
// zero for the next step.
template <int NT>
__device__ void spread_tiles(const Arrays &a, uint32_t gen, int cur, int bid, int nb, SpreadSmem &sm)
{
    static_assert(NT >= 16 * SPREAD_PARTS && NT >= TILE_CELLS, "a thread per part and x-row, and per cell");
    static_assert(TILE_CAP % NT == 0, "whole key passes");
    constexpr int HK = TILE_CAP / NT;              // a tile's nodes per thread, at most
    const int tid = threadIdx.x;
    const int nact = min(a.n_active[cur], a.active_cap);
    const int2 *list = a.active + (int64_t)cur * a.active_cap;
    // a block's next tile is looked up while it works on the current one:
    // its list entry at once, its count and first key once the entry is in
    // (a thread's first key slot is loaded whatever the count: the tile's
    // list has TILE_CAP slots, and slots beyond the count are not used)
    int2 te_n = bid < nact ? list[bid] : make_int2(0, 0);
    int cnt_n = -1, key0_n = 0x7fffffff;
    for (int it = bid; it < nact; it += nb) {
        const int2 te = te_n;
        if (it + nb < nact)
            te_n = list[it + nb];
        const int64_t T = te.x;
        const int d = a.ndrops == 1 ? 0 : find_drop_tile(a.drops, a.ndrops, T);
        const Drop &D = a.drops[d];
        const int X0 = 4 * (te.y & 2047), Y0 = 4 * ((te.y >> 11) & 2047), Z0 = 4 * (te.y >> 22);
        const int64_t e0 = T * TILE_CAP;
        // (overflow was flagged by the force kernel)
        const int cnt = min(cnt_n >= 0 ? cnt_n : a.bin_cnt[T], TILE_CAP);
        int key[HK];
#pragma unroll
        for (int h = 0; h < HK; ++h) {
            const int e = tid + h * NT;
            key[h] = 0x7fffffff;
            if (e < cnt) {
                key[h] = (h == 0 && cnt_n >= 0) ? key0_n : a.tile_list[e0 + e];
                sm.node[e] = key[h];
            }
        }
        if (tid < ((cnt + 3) & ~3) - cnt)
            sm.node[cnt + tid] = 0x7fffffff;             // pad the keys to a multiple of 4
        __syncthreads();
        if (tid == 0)
            a.bin_cnt[T] = 0;                            // empty for the next step
        int rank[HK];
        const int4 *keys4 = reinterpret_cast<const int4 *>(sm.node);
#pragma unroll
        for (int h = 0; h < HK; ++h) {
            rank[h] = -1;
            if (tid + h * NT < cnt) {
                int r = 0;
                for (int k = 0; k < (cnt + 3) >> 2; ++k) {
                    const int4 kv = keys4[k];
                    r += (kv.x < key[h]) + (kv.y < key[h]) + (kv.z < key[h]) + (kv.w < key[h]);
                }
                rank[h] = r;
            }
        }
        if (it + nb < nact) {   // the next tile's count and first key
            cnt_n = a.bin_cnt[te_n.x];
            key0_n = a.tile_list[(int64_t)te_n.x * TILE_CAP + tid];
        }
        // part sums: thread t < 16 SPREAD_PARTS takes part t / 16 of the
        // four cells of x-row t % 16 (y = row & 3, z = row >> 2 in the tile),
        // one load of the x weights serving the four cells
        const bool summer = tid < 16 * SPREAD_PARTS;
        const int part = (tid >> 4) & (SPREAD_PARTS - 1), row = tid & 15, ry = row & 3, rz = row >> 2;
        const int k0 = (int)(((int64_t)cnt * part) / SPREAD_PARTS);
        const int k1 = (int)(((int64_t)cnt * (part + 1)) / SPREAD_PARTS);
        float fx[4] = {0.f, 0.f, 0.f, 0.f}, fy[4] = {0.f, 0.f, 0.f, 0.f}, fz[4] = {0.f, 0.f, 0.f, 0.f};
        for (int w0 = 0; w0 < cnt; w0 += SPREAD_STAGE) {
            if (w0 > 0)
                __syncthreads();                         // the previous window's sums are done
#pragma unroll
            for (int h = 0; h < HK; ++h) {
                if (rank[h] >= w0 && rank[h] < w0 + SPREAD_STAGE) {
                    const NodeRec &r = a.rec[key[h]];
                    float wl[16];
                    tile_weights(X0, r.bx, D.nx, true, r.wx, wl);
                    tile_weights(Y0, r.by, D.ny, true, r.wy, wl + 4);
                    tile_weights(Z0, r.bz, D.nzf, !D.walls, r.wz, wl + 8);
                    wl[12] = r.phi[0];
                    wl[13] = r.phi[1];
                    wl[14] = r.phi[2];
                    wl[15] = 0.0f;
                    float4 *dst = reinterpret_cast<float4 *>(sm.rec[rank[h] - w0]);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_float4(wl[4 * q], wl[4 * q + 1], wl[4 * q + 2], wl[4 * q + 3]);
                }
            }
            __syncthreads();
            if (summer) {
                const int ka = max(k0, w0), kb = min(k1, w0 + SPREAD_STAGE);
                for (int k = ka; k < kb; ++k) {
                    const float *r = sm.rec[k - w0];
                    const float4 wx = *reinterpret_cast<const float4 *>(r);
                    const float wy = r[4 + ry], wz = r[8 + rz];
                    const float4 ph = *reinterpret_cast<const float4 *>(r + 12);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float w = ((&wx.x)[c] * wy) * wz;
                        fx[c] = fmaf(ph.x, w, fx[c]);
                        fy[c] = fmaf(ph.y, w, fy[c]);
                        fz[c] = fmaf(ph.z, w, fz[c]);
                    }
                }
            }
        }
        if (summer) {
            *reinterpret_cast<float4 *>(&sm.part[0][part][4 * row]) = make_float4(fx[0], fx[1], fx[2], fx[3]);
            *reinterpret_cast<float4 *>(&sm.part[1][part][4 * row]) = make_float4(fy[0], fy[1], fy[2], fy[3]);
            *reinterpret_cast<float4 *>(&sm.part[2][part][4 * row]) = make_float4(fz[0], fz[1], fz[2], fz[3]);
        }
        __syncthreads();
        const int cell = tid & (TILE_CELLS - 1), lane_part = tid / TILE_CELLS;
        const int X = X0 + (cell & 3), Y = Y0 + ((cell >> 2) & 3), Z = Z0 + (cell >> 4);
        if (lane_part == 0 && X < D.nx && Y < D.ny && Z < D.nzf) {
            float sx = sm.part[0][0][cell], sy = sm.part[1][0][cell], sz = sm.part[2][0][cell];
            for (int p = 1; p < SPREAD_PARTS; ++p) {
                sx += sm.part[0][p][cell];
                sy += sm.part[1][p][cell];
                sz += sm.part[2][p][cell];
            }
            const int64_t g = D.pcell0 + X + (int64_t)D.pitch * (Y + (int64_t)D.ny * Z);
            a.F[g] = sx;
            a.F[a.total_pcells + g] = sy;
            a.F[2 * a.total_pcells + g] = sz;
        }
        __syncthreads();
    }
}

// The last block to finish the spread commits the generation and empties the
// previous step's band list, which the next step fills.  A relaxed count
// suffices: the last block writes only these step-level words and reads
// nothing another block wrote, every block has read the generation and the
// previous band list before it counts, and the next kernel sees all the
// spread's writes at the kernel boundary (a release here made each block
// wait for its force-density stores first).
__device__ void spread_finish(const Arrays &a, uint32_t gen, int cur, SpreadSmem &sm)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        sm.last = cuda::atomic_ref<int, cuda::thread_scope_device>(*a.spread_done).fetch_add(
                      1, cuda::memory_order_relaxed) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (sm.last && threadIdx.x == 0) {
        *a.gen = gen;
        a.n_active[cur ^ 1] = 0;
        *a.spread_done = 0;
        *a.split_ok = 1;        // this band predicts the next step's
        a.grp_cnt[2] = 0;
    }
}

// Interpolation and advection of the IB_THREADS / 16 nodes of one block
// (base: the global index of its thread 0, a multiple of IB_THREADS).
// 16 lanes per node: lane l covers support row (dy, dz) = (l & 3, l >> 2)
// and the four cells of that row; partial sums meet in a fixed shuffle tree.
// The FP64 advection then runs on the block's first 3 IB_THREADS / 16
// threads, one coordinate each, so that its FP64 operations fill whole
// warps (on this GPU they issue at a small fraction of the FP32 rate); each
// thread reads its (corrected) coordinate when the kernel starts.
__device__ __forceinline__ void interp_block(const Arrays &a, int64_t base)
{
    constexpr int NPB = IB_THREADS / 16;
    __shared__ float inc_s[3 * NPB];
    const int64_t gid = base + threadIdx.x;
    const int j = (int)(gid >> 4), l = (int)(gid & 15);
    const bool valid = j < a.total_nodes;
    const int jn = (int)(base >> 4) + (int)threadIdx.x / 3, an = (int)threadIdx.x % 3;
    const bool adv = threadIdx.x < 3 * NPB && jn < a.total_nodes;
    double q = 0.0;
    if (adv)
        q = (an == 0 ? a.px : (an == 1 ? a.py : a.pz))[jn];
    float ax = 0.f, ay = 0.f, az = 0.f;
    int d = 0;
    if (valid) {
        d = a.ndrops == 1 ? 0 : a.node_drop[j];
        const NodeRec &r = a.rec[j];
        const Drop &D = a.drops[d];
        if (r.key > 0) {
            const int dy = l & 3, dz = l >> 2;
            int Z = r.bz - 1 + dz;
            bool fluid = true;
            if (D.walls)
                fluid = Z >= 0 && Z < D.nzf;
            else
                Z = wrapi(Z, D.nzf);
            if (fluid) {
                const int Y = wrapi(r.by - 1 + dy, D.ny);
                const float wyz = r.wy[dy] * r.wz[dz];
                const int64_t row = D.pcell0 + (int64_t)D.pitch * (Y + (int64_t)D.ny * Z);
                for (int dx = 0; dx < 4; ++dx) {
                    const int64_t g = row + wrapi(r.bx - 1 + dx, D.nx);
                    const float w = r.wx[dx] * wyz;
                    const float4 u = a.U[g];
                    ax = fmaf(u.x, w, ax);
                    ay = fmaf(u.y, w, ay);
                    az = fmaf(u.z, w, az);
                }
            }
        }
    }
    for (int o = 8; o >= 1; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (valid && l == 0) {
        if (!(isfinite(ax) && isfinite(ay) && isfinite(az)))
            atomicOr(&a.status[4 * d], ST_NAN);
        else if (ax * ax + ay * ay + az * az > 0.25f)
            atomicOr(&a.status[4 * d], ST_JUMP);
        float *o = inc_s + 3 * (j - (int)(base >> 4));
        o[0] = ax;
        o[1] = ay;
        o[2] = az;
    }
    __syncthreads();
    if (adv) {
        const double qn = q + (double)inc_s[threadIdx.x];
        (an == 0 ? a.qx : (an == 1 ? a.qy : a.qz))[jn] = qn;
        const float hi = dtof_rn(qn);
        reinterpret_cast<float *>(a.qh + jn)[an] = hi;
        reinterpret_cast<float *>(a.ql + jn)[an] = dtof_rn(qn - (double)hi);
    }
}

__device__ __forceinline__ int find_drop_chunk(const Drop *D, int n, int c)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].red_chunk0 <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Volume-correction chunk c (one block of VC_RB threads): faces and nodes
// [k*VC_RB, (k+1)*VC_RB) of its droplet (k = c - chunk0) give 6V and the
// node-coordinate sums; the chunk that finishes its droplet last folds the
// droplet's chunks in a fixed order and stores
// red_out = {(V0/V)^(1/3), cx, cy, cz, V}.
// Sums of NV values over the NT threads of a block, in a fixed order: the
// values go to shared memory, lane l of warp 0 adds entries l, l + 32, ...
// and the warp's lanes are combined by a shuffle tree.  Few FP64
// instructions (a warp-wide FP64 instruction is slow on this GPU).  Result
// in thread 0.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double *v)
{
    static_assert(NV * 32 <= NT, "one warp per value");
    __shared__ double sh[NV][NT];
    __shared__ double res[NV];
    for (int k = 0; k < NV; ++k)
        sh[k][threadIdx.x] = v[k];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < NV) {           // warp w sums value w
        double x = sh[w][lane];
        for (int i = lane + 32; i < NT; i += 32)
            x += sh[w][i];
        x = warp_sum(x);
        if (lane == 0)
            res[w] = x;
    }
    __syncthreads();
    for (int k = 0; k < NV; ++k)
        v[k] = res[k];
}

// (V/V0)^(-1/3) for s = V/V0 given as e = s - 1: the binomial series
// 1 - e/3 + 2e^2/9 - 14e^3/81 + 35e^4/243 - 91e^5/729 when |e| <= 2^-10
// (the first omitted term is below 1e-19, so the sum is within about one
// unit in the last place of the cube root), else cbrt(V0/V).  A step's
// volume drift is many orders below 2^-10; the series costs six dependent
// FP64 operations where the division and cube root cost about fifteen
// times as long on this GPU.
__device__ __forceinline__ double inv_cbrt_ratio(double e, double V0, double V)
{
    if (fabs(e) > 0x1p-10)
        return cbrt(V0 / V);
    double p = -91.0 / 729.0;
    p = fma(p, e, 35.0 / 243.0);
    p = fma(p, e, -14.0 / 81.0);
    p = fma(p, e, 2.0 / 9.0);
    p = fma(p, e, -1.0 / 3.0);
    return fma(p, e, 1.0);
}

// NT: the block size (at least VC_RB; threads beyond the chunk add zeros).
// WAIT: the launch follows the advection with programmatic dependent
// launch; the droplet lookup and the face corners (topology, which no step
// writes) are read before waiting for it, the positions after.
template <int NT, bool WAIT, bool TR = false>
__device__ void vc_chunk(const Arrays &a, int c, unsigned long long *tr = nullptr)
{
    static_assert(NT >= VC_RB, "a chunk needs VC_RB threads");
    __shared__ int s_last;
    const bool mine = threadIdx.x < VC_RB, one = a.ndrops == 1;
    int ia = 0, ib = 0, ic = 0;
    bool face = false;
    if (one) {      // one droplet: its faces and chunks start at 0, no droplet field is needed first
        const int t = c * VC_RB + threadIdx.x;
        face = mine && t < a.total_tri;
        if (face) {
            const int *f = a.tri + 3 * (int64_t)t;
            ia = f[0];
            ib = f[1];
            ic = f[2];
        }
    }
    const int d = find_drop_chunk(a.drops, a.ndrops, c);
    const Drop &D = a.drops[d];
    if (D.nnodes == 0 || !D.volcorr) {                 // block-uniform
        if (WAIT)
            griddep_wait();    // every block waits: the next launch may then read the advected positions
        return;
    }
    const int k = c - D.red_chunk0;
    const int t = k * VC_RB + threadIdx.x;
    const bool node = mine && t < D.nnodes;
    if (!one) {
        face = mine && t < D.ntri;
        if (face) {
            const int *f = a.tri + 3 * ((int64_t)D.tri0 + t);
            ia = f[0];
            ib = f[1];
            ic = f[2];
        }
    }
    if (WAIT) {
        griddep_wait();
        if constexpr (TR)
            trace_start(tr, TR_VC);
    }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (face) {   // 6 x the signed volume of the tetrahedron (0, q_a, q_b, q_c): q_a . (q_b x q_c)
        const double ax = a.qx[ia], ay = a.qy[ia], az = a.qz[ia];
        const double bx = a.qx[ib], by = a.qy[ib], bz = a.qz[ib];
        const double cx = a.qx[ic], cy = a.qy[ic], cz = a.qz[ic];
        const double x = fma(by, cz, -(bz * cy)), y = fma(bz, cx, -(bx * cz)), z = fma(bx, cy, -(by * cx));
        v[0] = fma(ax, x, fma(ay, y, az * z));
    }
    if (node) {
        const int j = D.node0 + t;
        v[1] = a.qx[j];
        v[2] = a.qy[j];
        v[3] = a.qz[j];
    }
    block_sum<4, NT>(v);
    double *part = a.red_part + (int64_t)NRED * c;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i)
            part[i] = v[i];
        // release: the partials above are visible to whoever sees the count
        s_last = cuda::atomic_ref<int, cuda::thread_scope_device>(a.vc_done[d]).fetch_add(
                     1, cuda::memory_order_acq_rel) == D.red_nchunks - 1;
    }
    __syncthreads();
    __shared__ double fold[4];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (s_last && w < 4) {
        // warp q folds value q of every chunk of the droplet: lane l adds
        // chunks l, l + 32, ... in that order.  Thread 0's acquire and the
        // block barrier order these loads after every chunk's release; they
        // read L2 (not the non-coherent L1), all of a pass issued at once.
        constexpr int U = 8;
        const double *pp = a.red_part + (int64_t)NRED * D.red_chunk0 + w;
        double x = 0.0;
        for (int i0 = lane; i0 < D.red_nchunks; i0 += 32 * U) {
            double t[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + 32 * u;
                t[u] = i < D.red_nchunks ? __ldcg(pp + (int64_t)NRED * i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                x += t[u];
        }
        x = warp_sum(x);
        if (lane == 0)
            fold[w] = x;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 4) {
        // lane 0: V = fold0 / 6 and k = (V0/V)^(1/3); lanes 1-3: the centroid
        double *o = a.red_out + (int64_t)NRED * d;
        const double f = fold[threadIdx.x];
        if (threadIdx.x == 0) {
            const double V = f * (1.0 / 6.0);
            o[0] = inv_cbrt_ratio(fma(f, D.inv6V0, -1.0), D.V0, V);
            o[4] = V;
            o[5] = 1.0;     // applied wherever the positions are read next
            a.vc_done[d] = 0;
        } else {
            o[threadIdx.x] = f * D.inv_n;
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------- grid barrier
// Sense-reversing barrier over the blocks of a cooperative launch (all of
// them resident).  `sense` is thread 0's copy of the release flag, read once
// when the kernel starts.  The wait is bounded: a block that gives up flags
// ST_TIMEOUT and returns false, and its caller leaves the kernel.
__device__ bool grid_barrier(const Arrays &a, unsigned &sense)
{
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_fail = 0;
        sense ^= 1u;
        __threadfence();
        if (atomicAdd(a.bar_count, 1u) == gridDim.x - 1) {
            *a.bar_count = 0;
            __threadfence();
            atomicExch(a.bar_flag, sense);
        } else {
            const long long t0 = clock64();
            while (*(volatile unsigned *)a.bar_flag != sense) {
                if (clock64() - t0 > BARRIER_CYCLES) {
                    s_fail = 1;
                    atomicOr(&a.status[0], ST_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return !s_fail;
}

// ------------------------------------------------------------------ kernels
constexpr int NF_THREADS = 64;   // block size of the force kernel (16 nodes): small blocks, so that a
                                 // mesh of ten thousand nodes spreads evenly over every SM (641
                                 // blocks; 128-thread blocks measured 0.1-0.3 us slower per step)

template <bool EL, bool TR>
__global__ void __launch_bounds__(NF_THREADS) node_force_kernel(Arrays a, unsigned long long *tr)
{
    griddep_wait();
    if constexpr (TR)
        trace_start(tr, TR_FORCE);
    const uint32_t gen = *a.gen + 1u;                  // committed by the spread
    node_forces<EL>(a, (int64_t)blockIdx.x * NF_THREADS + threadIdx.x, gen);
}

template <bool TR>
__global__ void __launch_bounds__(SP_THREADS, SP_PER_SM) spread_kernel(Arrays a, unsigned long long *tr)
{
    griddep_wait();
    if constexpr (TR)
        trace_start(tr, TR_SPREAD);
    __shared__ SpreadSmem sm;
    const uint32_t gen = *a.gen + 1u;
    const int cur = (int)(gen & 1u);
    const LeftTile first = zero_left_first<SP_THREADS>(a, cur, blockIdx.x);
    spread_tiles<SP_THREADS>(a, gen, cur, blockIdx.x, gridDim.x, sm);
    zero_left_tiles<SP_THREADS>(a, gen, cur, blockIdx.x, gridDim.x, first);
    spread_finish(a, gen, cur, sm);
}

template <bool TR>
__global__ void __launch_bounds__(IB_THREADS) interp_advect_kernel(Arrays a, unsigned long long *tr)
{
    griddep_wait();
    if constexpr (TR)
        trace_start(tr, TR_INTERP);
    interp_block(a, (int64_t)blockIdx.x * IB_THREADS);
}

// The volume correction of every droplet: FP64 volume and centroid
// partials of chunk blockIdx.x; the last chunk of a droplet folds them into
// k = (V0/V)^(1/3) and the centroid, which the readers of the positions
// apply from then on.
template <bool TR>
__global__ void __launch_bounds__(VC_RB) volume_correction_kernel(Arrays a, unsigned long long *tr)
{
    vc_chunk<VC_RB, true, TR>(a, blockIdx.x, tr);
}

// The trailing marker of a traced step: starts once the step's last kernel
// has finished.
__global__ void trace_marker_kernel(Arrays a, unsigned long long *tr)
{
    griddep_wait();
    trace_start(tr, TR_END);
}

// a.p* = the positions as read (the pending correction applied)
// and, for nodes node0 .. node0 + n - 1 when xyz is set, the same
// positions interleaved (x, y, z per node) into xyz
__global__ void __launch_bounds__(IB_THREADS) corrected_positions_kernel(Arrays a, double *xyz, int node0, int n)
{
    griddep_wait();
    const int j = blockIdx.x * IB_THREADS + threadIdx.x;
    if (j >= a.total_nodes)
        return;
    double x = a.qx[j], y = a.qy[j], z = a.qz[j];
    const Corr cr = load_corr(a, a.node_drop[j]);
    if (cr.on) {
        x = corr1(x, cr.cx, cr.k);
        y = corr1(y, cr.cy, cr.k);
        z = corr1(z, cr.cz, cr.k);
    }
    a.px[j] = x;
    a.py[j] = y;
    a.pz[j] = z;
    if (xyz && j >= node0 && j < node0 + n) {
        double *o = xyz + 3 * (int64_t)(j - node0);
        o[0] = x;
        o[1] = y;
        o[2] = z;
    }
}

// Positions of droplet k's nodes node0 .. node0 + n - 1 from xyz (x, y, z
// per node), final (no volume correction pending for the droplet), with
// their FP32 pairs; the previous band no longer predicts this step's.
__global__ void __launch_bounds__(IB_THREADS) set_nodes_kernel(Arrays a, const double *xyz, int node0, int n, int k)
{
    const int j = blockIdx.x * IB_THREADS + threadIdx.x;
    if (j == 0) {
        a.red_out[(int64_t)NRED * k + 5] = 0.0;
        *a.split_ok = 0;
    }
    if (j >= n)
        return;
    const double *p = xyz + 3 * (int64_t)j;
    const double x = p[0], y = p[1], z = p[2];
    const int g = node0 + j;
    a.qx[g] = x;
    a.qy[g] = y;
    a.qz[g] = z;
    const float hx = dtof_rn(x), hy = dtof_rn(y), hz = dtof_rn(z);
    a.qh[g] = make_float4(hx, hy, hz, 0.0f);
    a.ql[g] = make_float4(dtof_rn(x - (double)hx), dtof_rn(y - (double)hy), dtof_rn(z - (double)hz), 0.0f);
}

// Before the stream-collide kernel: forces and tile lists of every node,
// grid barrier, spread of every band tile.
template <bool EL>
__global__ void __launch_bounds__(IB_THREADS) ib_front_kernel(Arrays a)
{
    __shared__ SpreadSmem sm;
    unsigned sense = *(volatile unsigned *)a.bar_flag;
    const uint32_t gen = *a.gen + 1u;
    const int cur = (int)(gen & 1u);
    const int64_t nf = ((int64_t)a.total_nodes * NL + 31) & ~(int64_t)31;   // whole warps
    const int64_t stride = (int64_t)gridDim.x * IB_THREADS;
    for (int64_t gid = (int64_t)blockIdx.x * IB_THREADS + threadIdx.x; gid < nf; gid += stride)
        node_forces<EL>(a, gid, gen);
    if (!grid_barrier(a, sense))
        return;
    const LeftTile first = zero_left_first<IB_THREADS>(a, cur, blockIdx.x);
    spread_tiles<IB_THREADS>(a, gen, cur, blockIdx.x, gridDim.x, sm);
    zero_left_tiles<IB_THREADS>(a, gen, cur, blockIdx.x, gridDim.x, first);
    spread_finish(a, gen, cur, sm);
}

// After the stream-collide kernel: interpolation and advection of every
// node; then, if some droplet corrects its volume, grid barrier, FP64 volume
// and centroid of every droplet (the correction stays pending).
__global__ void __launch_bounds__(IB_THREADS) ib_back_kernel(Arrays a, int n_chunks, int volcorr)
{
    unsigned sense = *(volatile unsigned *)a.bar_flag;
    const int64_t ni = (int64_t)a.total_nodes * 16;
    const int64_t stride = (int64_t)gridDim.x * IB_THREADS;
    for (int64_t base = (int64_t)blockIdx.x * IB_THREADS; base < ni; base += stride) {   // block-uniform
        interp_block(a, base);
        __syncthreads();    // the next pass rewrites inc_s
    }
    if (!volcorr)
        return;
    if (!grid_barrier(a, sense))
        return;
    for (int c = blockIdx.x; c < n_chunks; c += gridDim.x)
        vc_chunk<IB_THREADS, false>(a, c);
}

int g_sm_count = 0;
int g_front_blocks[2] = {0, 0}, g_back_blocks = 0;

int sm_count()
{
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    return g_sm_count;
}

}  // namespace

cudaError_t launch_node_force(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    const dim3 grid((unsigned)(((int64_t)a.total_nodes * NL + NF_THREADS - 1) / NF_THREADS));
    if (a.fref)
        return g_trace_ib ? launch_k(node_force_kernel<true, true>, grid, dim3(NF_THREADS), 0, s, a.pdl != 0, a,
                                     g_trace_ib)
                          : launch_k(node_force_kernel<true, false>, grid, dim3(NF_THREADS), 0, s, a.pdl != 0, a,
                                     (unsigned long long *)nullptr);
    return g_trace_ib ? launch_k(node_force_kernel<false, true>, grid, dim3(NF_THREADS), 0, s, a.pdl != 0, a,
                                 g_trace_ib)
                      : launch_k(node_force_kernel<false, false>, grid, dim3(NF_THREADS), 0, s, a.pdl != 0, a,
                                 (unsigned long long *)nullptr);
}

cudaError_t launch_spread(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    const dim3 grid(sm_count() * SP_PER_SM);
    return g_trace_ib ? launch_k(spread_kernel<true>, grid, dim3(SP_THREADS), 0, s, a.pdl != 0, a, g_trace_ib)
                      : launch_k(spread_kernel<false>, grid, dim3(SP_THREADS), 0, s, a.pdl != 0, a,
                                 (unsigned long long *)nullptr);
}

void set_trace_ib(unsigned long long *trace) { g_trace_ib = trace; }

cudaError_t launch_trace_marker(const Arrays &a, unsigned long long *trace, cudaStream_t s)
{
    return launch_k(trace_marker_kernel, dim3(1), dim3(32), 0, s, a.pdl != 0, a, trace);
}

cudaError_t launch_interp_advect(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    const int64_t threads = (int64_t)a.total_nodes * 16;
    const dim3 grid((unsigned)((threads + IB_THREADS - 1) / IB_THREADS));
    return g_trace_ib ? launch_k(interp_advect_kernel<true>, grid, dim3(IB_THREADS), 0, s, a.pdl != 0, a, g_trace_ib)
                      : launch_k(interp_advect_kernel<false>, grid, dim3(IB_THREADS), 0, s, a.pdl != 0, a,
                                 (unsigned long long *)nullptr);
}


// Cooperative launches: every block must be resident, so the grid is at
// most the number of blocks that fit on the device at once; per_sm > 0 asks
// for fewer (a grid barrier over fewer blocks is cheaper), and the grid never
// exceeds what the work needs.
static cudaError_t coop_grid(const void *fn, int64_t want, int per_sm_req, int &grid, int &cache)
{
    if (!cache) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, IB_THREADS, 0);
        if (e != cudaSuccess)
            return e;
        if (per_sm < 1)
            return cudaErrorInvalidConfiguration;
        cache = per_sm;
    }
    const int per_sm = per_sm_req > 0 && per_sm_req < cache ? per_sm_req : cache;
    const int64_t cap = (int64_t)per_sm * sm_count();
    grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    return cudaSuccess;
}

cudaError_t launch_ib_front(const Arrays &a, int per_sm, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    int grid = 0;
    const int64_t want = ((int64_t)a.total_nodes * NL + IB_THREADS - 1) / IB_THREADS;
    const bool el = a.fref != nullptr;
    const void *fn = el ? (const void *)ib_front_kernel<true> : (const void *)ib_front_kernel<false>;
    cudaError_t e = coop_grid(fn, std::max<int64_t>(want, (int64_t)sm_count()), per_sm, grid, g_front_blocks[el]);
    if (e != cudaSuccess)
        return e;
    Arrays arg = a;
    void *args[] = {&arg};
    return cudaLaunchCooperativeKernel(fn, grid, IB_THREADS, args, 0, s);
}

cudaError_t launch_volume_correction(const Arrays &a, int n_chunks_total, cudaStream_t s)
{
    if (a.total_nodes <= 0 || n_chunks_total <= 0)
        return cudaSuccess;
    return g_trace_ib ? launch_k(volume_correction_kernel<true>, dim3(n_chunks_total), dim3(VC_RB), 0, s,
                                 a.pdl != 0, a, g_trace_ib)
                      : launch_k(volume_correction_kernel<false>, dim3(n_chunks_total), dim3(VC_RB), 0, s,
                                 a.pdl != 0, a, (unsigned long long *)nullptr);
}

cudaError_t launch_corrected_positions(const Arrays &a, cudaStream_t s, double *xyz, int node0, int n)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    return launch_k(corrected_positions_kernel, dim3((a.total_nodes + IB_THREADS - 1) / IB_THREADS),
                    dim3(IB_THREADS), 0, s, a.pdl != 0, a, xyz, node0, n);
}

cudaError_t launch_set_nodes(const Arrays &a, const double *xyz, int node0, int n, int k, cudaStream_t s)
{
    set_nodes_kernel<<<(n + IB_THREADS - 1) / IB_THREADS, IB_THREADS, 0, s>>>(a, xyz, node0, n, k);
    return cudaGetLastError();
}

cudaError_t launch_ib_back(const Arrays &a, int n_chunks_total, bool volcorr, int per_sm, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    int grid = 0;
    const int64_t want = ((int64_t)a.total_nodes * 16 + IB_THREADS - 1) / IB_THREADS;
    cudaError_t e = coop_grid((const void *)ib_back_kernel, std::max<int64_t>(want, n_chunks_total), per_sm, grid,
                              g_back_blocks);
    if (e != cudaSuccess)
        return e;
    Arrays arg = a;
    int nc = n_chunks_total, vc = volcorr ? 1 : 0;
    void *args[] = {&arg, &nc, &vc};
    return cudaLaunchCooperativeKernel((const void *)ib_back_kernel, grid, IB_THREADS, args, 0, s);
}

}  // namespace iblb
