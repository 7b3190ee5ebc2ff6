// lb.cu -- fused pull-stream + halfway bounce-back + moments + BGK + Guo
// source for D3Q19 (Sec. II A: eqs. LBE, hydro_var1, hydro_var2, the BGK
// operator, the equilibrium and Guo's source term), populations stored as
// offsets s_i = f_i - w_i rho0 in FP32, FP16 or BF16, arithmetic in FP32.
//
// Data movement.  Populations and the force / velocity fields live in rows
// (y, z) of pitch P (nx rounded up to 16 elements), so every row starts on a
// 32-byte boundary.  A group is R consecutive cell rows of one droplet.  In
// the pull scheme population i of row (y, z) comes entirely from row
// (y - c_iy, z - c_iz) (or, at a wall, from row (y, z) of the opposite
// population), so one producer warp per block fetches the 19 R source rows of
// a group -- plus the three force-density rows of every row that meets the
// band around the membrane -- into shared memory with TMA bulk copies
// (cp.async.bulk, completion on an mbarrier), and the eight consumer warps
// apply the x shift and the periodic x wrap inside shared memory.  Every
// population row is read from HBM exactly once per step; the consumers
// touch global memory only to store results.  Blocks are persistent and
// keep a ring of 2 to 8 stages with a pair of mbarriers each: "full" (the
// bulk copies landed) and "empty" (every consumer thread finished reading).
// The producer refills a stage as soon as it is empty, so up to ns groups
// are in flight, and no consumer warp waits for the others.
//
// Memory traffic per fluid cell: 19 reads + 19 writes of the storage type
// (152 B for FP32, 76 B for 16-bit storage); the force density is read and
// the velocity written only on band rows.
#include <algorithm>

#include "iblb_internal.h"
#include "mbarrier.cuh"

namespace iblb {

namespace {

unsigned long long *g_trace_lb = nullptr;   // host: stamp buffer of a traced step (see iblb_trace_step)
// The traced kernel's stamp as a call: inlined, it costs the collision loop
// a register spill, and the traced step would not time the plain kernel.
__device__ __noinline__ void lb_trace_start(unsigned long long *tr) { trace_start(tr, TR_LB); }

constexpr int LB_THREADS = 256;                   // consumer threads per block (FP32 storage)
// 16-bit storage takes two cells per work item and needs more registers per
// thread: 7 consumer warps (+ the producer) keep two blocks of 8 warps on an
// SM at up to 128 registers, where two blocks of 9 warps allow 96
template <typename S>
constexpr int cons_threads() { return sizeof(S) == 2 ? 224 : LB_THREADS; }
template <typename S>
constexpr int lb_block() { return cons_threads<S>() + 32; }   // + one producer warp
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz: bounded mbarrier wait
constexpr int LB_MAX_STAGES = 8;

__device__ __forceinline__ float cvt(float v) { return v; }
__device__ __forceinline__ float cvt(__half v) { return __half2float(v); }
__device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
// population stores are streamed (evict-first in L2): they are read again
// only in the next step
__device__ __forceinline__ void st(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st(__half *p, float v) { __stcs(p, __float2half_rn(v)); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { __stcs(p, __float2bfloat16_rn(v)); }

__device__ __forceinline__ int find_drop_group(const Drop *D, int n, int g)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].lb_block0 <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}


__constant__ int kCy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int kCz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
__constant__ int kOpp[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};

constexpr float W0 = 1.0f / 3.0f, W1 = 1.0f / 18.0f, W2 = 1.0f / 36.0f;
// Coefficients 3 w of the first-order (odd) part, chosen so that the
// lattice isotropy sum 2 K1 + 8 K2 = sum_i 3 w_i c_ix^2 is exactly 1 in FP32
// arithmetic: K2 = fl(1/12), K1 = (1 - 8 K2) / 2 (both exact).  With
// fl(3 w) for each class the sum is 1 + 2^-25, and every collision would
// scale the momentum by 1 + omega 2^-25: in a uniform stream every cell
// rounds alike and that gain adds up step after step.
constexpr float K2 = 1.0f / 12.0f, K1 = (1.0f - 8.0f * K2) * 0.5f;

// stage layout: [19][R][P] populations | [3][R][P] force | band flag
template <typename S>
struct Stage {
    S *pop;
    float *F;
    int *flag;
    __device__ Stage(unsigned char *base, int R, int P)
    {
        pop = reinterpret_cast<S *>(base);
        F = reinterpret_cast<float *>(base + (size_t)R * Q * P * sizeof(S));
        flag = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(F) + (size_t)R * 3 * P * sizeof(float));
    }
};

// rows y0 .. y0 + nr - 1 of plane z in group g of droplet D
__device__ __forceinline__ void group_rows(const Drop &D, int g, int &y0, int &z, int &nr)
{
    const int lg = g - D.lb_block0;
    z = lg / D.lb_gpp;
    y0 = (lg - z * D.lb_gpp) * D.lb_rows;
    nr = min(D.lb_rows, D.ny - y0);
}

// A droplet's stream-collide constants, loaded once and kept in registers
// while consecutive groups of the same droplet run (one droplet per launch
// is the common case), with the thread's first cell (r0, x0) of a group.
struct DropC {
    int d, nx, ny, P, R, PC, nzf, walls, vartau, gpp, block0, step_r, step_x, r0, x0;
    int npr, pstep_r, pstep_x, pr0, px0;   // the same walk over cell pairs (x, x + 1), x even
    int tx, ty;                            // tiles per row and per plane of tile rows
    int64_t tile0;
    float inv_gpp, bfx, bfy, bfz, rho0, omega_out, omega_in;
    bool has_bf;
    int64_t pcell0, col0;
    __device__ __forceinline__ void load(const Drop &D, int dd, int nt)
    {
        d = dd;
        nx = D.nx;
        ny = D.ny;
        P = D.pitch;
        R = D.lb_rows;
        PC = (int)D.pcells;
        nzf = D.nzf;
        walls = D.walls;
        vartau = D.vartau;
        gpp = D.lb_gpp;
        block0 = D.lb_block0;
        step_r = nt / nx;
        step_x = nt - step_r * nx;
        r0 = threadIdx.x / nx;
        x0 = threadIdx.x - r0 * nx;
        tx = D.tx;
        ty = D.ty;
        tile0 = D.tile0;
        npr = (nx + 1) >> 1;
        pstep_r = nt / npr;
        pstep_x = nt - pstep_r * npr;
        pr0 = threadIdx.x / npr;
        px0 = threadIdx.x - pr0 * npr;
        inv_gpp = 1.0f / (float)gpp;
        bfx = D.bf[0];
        bfy = D.bf[1];
        bfz = D.bf[2];
        rho0 = D.rho0;
        omega_out = D.omega_out;
        omega_in = D.omega_in;
        has_bf = bfx != 0.0f || bfy != 0.0f || bfz != 0.0f;
        pcell0 = D.pcell0;
        col0 = D.col0;
    }
    // rows y0 .. y0 + nr - 1 of plane z in group g (as group_rows, without
    // an integer division: a float estimate of the quotient, corrected once)
    __device__ __forceinline__ void rows(int g, int &y0, int &z, int &nr) const
    {
        const int lg = g - block0;
        z = (int)((float)lg * inv_gpp);
        int rem = lg - z * gpp;
        if (rem < 0) {
            --z;
            rem += gpp;
        } else if (rem >= gpp) {
            ++z;
            rem -= gpp;
        }
        y0 = rem * R;
        nr = min(R, ny - y0);
    }
};

// Band flags of 32 consecutive groups of a block, one per lane: lane l
// takes group ig0 + l * stride.  A group carries force iff one of the tile
// rows its cell rows cross put a tile into this step's band (the force
// kernel stamps the row with the step's generation; F vanishes outside band
// tiles).  Bit l of the result is lane l's flag.
__device__ __forceinline__ uint32_t band_ballot(const Arrays &a, const int *list, int total, int ig0, int stride,
                                                uint32_t gen)
{
    const int lane = threadIdx.x & 31;
    const int ig = ig0 + lane * stride;
    bool band = false;
    if (ig < total) {
        const int g = list ? list[ig] : ig;
        const Drop &D = a.drops[find_drop_group(a.drops, a.ndrops, g)];
        int y0, z, nr;
        group_rows(D, g, y0, z, nr);
        const int64_t tr0 = D.trow0 + (int64_t)D.ty * (z >> 2);
        for (int ty = y0 >> 2; ty <= (y0 + nr - 1) >> 2; ++ty)
            band |= a.rowgen[tr0 + ty] == gen;
    }
    return __ballot_sync(0xffffffffu, band);
}

// Producer warp: fetch group g into a stage.  The source rows of population i
// for rows y0 .. y0+nr-1 of plane z are rows y0-c_iy .. of plane z-c_iz
// (or the group's own rows of the opposite population at a wall), which are
// contiguous in memory except across the periodic y seam: lane i < 19 issues
// one bulk copy for population i (two at the seam).  If the group carries
// force (band), lanes 19..21 copy the three force-density components of the
// group's rows.  Every lane announces the bytes of its own copies on the
// mbarrier (initialised for 32 arrivals) before issuing them.
template <typename S>
__device__ __forceinline__ void produce(const Arrays &a, const DropC &c, const S *src, int y0, int z, int nr,
                                        unsigned char *sbase, uint64_t *bar, bool band)
{
    const int lane = threadIdx.x & 31;
    const int P = c.P, ny = c.ny, R = c.R;
    Stage<S> stg(sbase, R, P);
    const int64_t plane_row0 = (int64_t)ny * z;
    const uint32_t rowb = (uint32_t)(P * sizeof(S));
    // copies of this lane: up to two pieces (source row, destination row, rows)
    int src_pop = 0, src_z = 0, y_a = 0, n_a = 0, y_b = 0, n_b = 0, d_b = 0;
    uint32_t mine = 0;
    if (lane < Q) {
        const int i = lane;
        int zs = z - kCz[i], ys = y0 - kCy[i];
        src_pop = i;
        if (c.walls && (zs < 0 || zs >= c.nzf)) {
            src_pop = kOpp[i];          // halfway bounce-back: own rows, opposite population
            zs = z;
            ys = y0;
        } else {
            zs = wrapi(zs, c.nzf);
        }
        src_z = zs;
        if (ys < 0) {                   // first row wraps to y = ny - 1
            y_a = ny - 1; n_a = 1;
            y_b = 0; n_b = nr - 1; d_b = 1;
        } else if (ys + nr > ny) {      // last row wraps to y = 0
            y_a = ys; n_a = ny - ys;
            y_b = 0; n_b = nr - n_a; d_b = n_a;
        } else {
            y_a = ys; n_a = nr;
        }
        mine = rowb * (uint32_t)(n_a + n_b);
    } else if (band && lane < Q + 3) {
        mine = (uint32_t)(nr * P * sizeof(float));
    }
    if (lane == 0)
        *stg.flag = band;
    mbar_arrive_expect_tx(bar, mine);
    if (lane < Q) {
        const S *plane = src + (int64_t)Q * c.pcell0 + (int64_t)src_pop * c.PC + (int64_t)P * ny * src_z;
        S *dst = stg.pop + (int64_t)lane * R * P;
        const uint64_t pol = l2_evict_first();
        if (n_a > 0)
            bulk_g2s_hint(dst, plane + (int64_t)P * y_a, rowb * n_a, bar, pol);
        if (n_b > 0)
            bulk_g2s_hint(dst + (int64_t)d_b * P, plane + (int64_t)P * y_b, rowb * n_b, bar, pol);
    } else if (band && lane < Q + 3) {
        const int k = lane - Q;
        bulk_g2s(stg.F + (int64_t)k * R * P, a.F + k * a.total_pcells + c.pcell0 + (int64_t)P * (plane_row0 + y0),
                 (uint32_t)(nr * P * sizeof(float)), bar);
    }
}

// BGK + Guo for one group's cells.  For the pair (i, opp(i)), c_opp = -c_i,
// with cu = c_i.U and cF = c_i.F the post-collision offsets
// s*_i = (1 - omega) s_i + omega s_eq_i + S_i  regroup as
//   s*_i   = (1 - omega) s_i   + P + M,
//   s*_opp = (1 - omega) s_opp + P - M,
//   P = w X + cu (9/2 w omega rho cu + 9 w k cF),   M = 3 w (omega rho cu + k cF),
//   X = omega (drho - 3/2 rho U.U) - 3 k U.F,         k = 1 - omega/2,
// (the equilibrium's even part w drho + w rho (9/2 cu^2 - 3/2 U.U) and odd
// part 3 w rho cu, Guo's source (1 - omega/2) w (3 (c_i - U) + 9 cu c_i).F),
// and the rest population is s*_0 = (1 - omega) s_0 + w_0 X.  FORCE false
// is the case F = 0 (a group outside the band without a body force), where
// every F term drops out; it rounds exactly as the FORCE path does with
// F = 0, so a cell's result does not depend on which group shape holds it.
// the cell's tile is in this step's band: its velocity is read by the
// interpolation (every node's kernel support lies in band tiles)
__device__ __forceinline__ bool in_band_tile(const Arrays &a, const DropC &c, int x, int y, int z, uint32_t gen)
{
    return a.tile_gen[c.tile0 + (x >> 2) + (int64_t)c.tx * ((y >> 2) + (int64_t)c.ty * (z >> 2))] == gen;
}

template <typename S, bool VARTAU, bool FORCE>
__device__ __forceinline__ void collide_group(const Arrays &a, const DropC &c, const Stage<S> &stg, int y0, int z,
                                              int nr, bool band, S *__restrict__ dst, uint32_t gen)
{
    const int nx = c.nx, ny = c.ny, P = c.P, R = c.R;
    const int PC = c.PC;
    const int64_t pcell0 = c.pcell0;
    const float bfx = c.bfx, bfy = c.bfy, bfz = c.bfz, rho0 = c.rho0;
    const float omega_out = c.omega_out, omega_in = c.omega_in;
    const int vartau = c.vartau, walls = c.walls;
    const int64_t col0 = c.col0;
    const bool bbm = walls && z == 0;              // rows pulled from z-1 bounced at the bottom
    const bool bbp = walls && z == c.nzf - 1;      // rows pulled from z+1 bounced at the top
    const int RP = R * P;
    S *outb = dst + (int64_t)Q * pcell0 + (int64_t)P * ny * z;
    float4 *U = a.U;
    // cell e = r * nx + x of the group, walked without divisions
    const int step_r = c.step_r, step_x = c.step_x;
    int r = c.r0, x = c.x0;
    for (; r < nr; r += step_r, x += step_x) {
        if (x >= nx) {
            x -= nx;
            ++r;
            if (r >= nr)
                break;
        }
        const int y = y0 + r;
        float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
        if (FORCE) {
            Fx = bfx;
            Fy = bfy;
            Fz = bfz;
            if (band) {     // F vanishes outside band tiles
                const float *Fr = stg.F + r * P + x;
                Fx += Fr[0];
                Fy += Fr[RP];
                Fz += Fr[2 * RP];
            }
        }
        float omega = omega_out;
        if (VARTAU && vartau) {
            const int64_t col = col0 + x + (int64_t)nx * y;
            const int cnt = min(a.col_cnt[col], MAXC);
            const double Z = (double)(z + walls);
            int par = 0;
            for (int q = 0; q < cnt; ++q)
                par ^= a.col_z[col * MAXC + q] < Z;
            if (par)
                omega = omega_in;
        }
        const int xm = x ? x - 1 : nx - 1, xp = x + 1 < nx ? x + 1 : 0;
        const S *Rr = stg.pop + r * P;
#define IN(i, xx) cvt(Rr[(i) * RP + (xx)])
        const float s0 = IN(0, x);
        const float s1 = IN(1, xm);
        const float s2 = IN(2, xp);
        const float s3 = IN(3, x);
        const float s4 = IN(4, x);
        const float s5 = IN(5, x);
        const float s6 = IN(6, x);
        const float s7 = IN(7, xm);
        const float s8 = IN(8, xp);
        const float s9 = IN(9, xm);
        const float s10 = IN(10, xp);
        const float s11 = IN(11, x);
        const float s12 = IN(12, x);
        const float s13 = IN(13, x);
        const float s14 = IN(14, x);
        const float s15 = IN(15, bbm ? x : xm);
        const float s16 = IN(16, bbp ? x : xp);
        const float s17 = IN(17, bbp ? x : xm);
        const float s18 = IN(18, bbm ? x : xp);
#undef IN
        // moments (eqs. hydro_var1, hydro_var2) in offset form, from the
        // sums and differences of opposite pairs
        const float p1 = s1 + s2, m1 = s1 - s2, p3 = s3 + s4, m3 = s3 - s4, p5 = s5 + s6, m5 = s5 - s6;
        const float p7 = s7 + s8, m7 = s7 - s8, p9 = s9 + s10, m9 = s9 - s10;
        const float p11 = s11 + s12, m11 = s11 - s12, p13 = s13 + s14, m13 = s13 - s14;
        const float p15 = s15 + s16, m15 = s15 - s16, p17 = s17 + s18, m17 = s17 - s18;
        const float drho = ((s0 + p1) + (p3 + p5)) + ((p7 + p9) + (p11 + p13)) + (p15 + p17);
        const float jx = ((m1 + m7) + (m9 + m15)) + m17;
        const float jy = ((m3 + m7) - (m9 - m11)) + m13;
        const float jz = ((m5 + m11) - (m13 - m15)) - m17;
        const float rho = rho0 + drho;
        const float irho = __fdividef(1.0f, rho);
        // J = rho U = j + F/2 (eq. hydro_var2)
        const float Jx = FORCE ? fmaf(0.5f, Fx, jx) : jx;
        const float Jy = FORCE ? fmaf(0.5f, Fy, jy) : jy;
        const float Jz = FORCE ? fmaf(0.5f, Fz, jz) : jz;
        const float ux = Jx * irho, uy = Jy * irho, uz = Jz * irho;
        const int64_t cell = (int64_t)P * (y + (int64_t)ny * z) + x;
        if (FORCE && band && in_band_tile(a, c, x, y, z, gen)) {
            const int64_t gi = pcell0 + cell;
            U[gi] = make_float4(ux, uy, uz, 0.0f);
        }
        const float om1 = 1.0f - omega, k = fmaf(-0.5f, omega, 1.0f), er = omega * rho;
        float X = omega * fmaf(-1.5f * rho, fmaf(ux, ux, fmaf(uy, uy, uz * uz)), drho);
        if (FORCE)
            X = fmaf(-3.0f * k, fmaf(ux, Fx, fmaf(uy, Fy, uz * Fz)), X);
        S *o = outb + P * y + x;
        st(o, fmaf(om1, s0, W0 * X));
        // per weight class: b = w X, ea = 9/2 w omega rho, kf = 9 w k for the
        // even part; the odd part takes 3 w omega rho (c.U) + 3 w k (c.F) as
        // ec (c.J) + kd (c.F) with ec = K omega, kd = K k, J = rho U, so that
        // the collision adds exactly (1 - omega/2) F to the momentum and
        // leaves the rest unchanged, up to the rounding of each result
        const float b1 = W1 * X, ea1 = (4.5f * W1) * er, ec1 = K1 * omega;
        const float b2 = W2 * X, ea2 = (4.5f * W2) * er, ec2 = K2 * omega;
        const float kf1 = (9.0f * W1) * k, kd1 = K1 * k, kf2 = (9.0f * W2) * k, kd2 = K2 * k;
#define PAIR(i, j, b, ea, ec, kf, kd, cu_e, cJ_e, cF_e, si, sj)                                           \
        {                                                                                                \
            const float cu_ = (cu_e), cJ_ = (cJ_e);                                                      \
            float Pp, Mm;                                                                                \
            if (FORCE) {                                                                                 \
                const float cF_ = (cF_e);                                                                \
                Mm = fmaf(ec, cJ_, kd * cF_);                                                            \
                Pp = fmaf(fmaf(ea, cu_, kf * cF_), cu_, b);                                              \
            } else { /* unfused products: the same roundings as with F = 0 above */                    \
                Mm = __fmul_rn(ec, cJ_);                                                                 \
                Pp = fmaf(__fmul_rn(ea, cu_), cu_, b);                                                   \
            }                                                                                            \
            st(o + (i) * PC, fmaf(om1, (si), Pp + Mm));                                                  \
            st(o + (j) * PC, fmaf(om1, (sj), Pp - Mm));                                                  \
        }
        PAIR(1, 2, b1, ea1, ec1, kf1, kd1, ux, Jx, Fx, s1, s2);
        PAIR(3, 4, b1, ea1, ec1, kf1, kd1, uy, Jy, Fy, s3, s4);
        PAIR(5, 6, b1, ea1, ec1, kf1, kd1, uz, Jz, Fz, s5, s6);
        PAIR(7, 8, b2, ea2, ec2, kf2, kd2, ux + uy, Jx + Jy, Fx + Fy, s7, s8);
        PAIR(9, 10, b2, ea2, ec2, kf2, kd2, ux - uy, Jx - Jy, Fx - Fy, s9, s10);
        PAIR(11, 12, b2, ea2, ec2, kf2, kd2, uy + uz, Jy + Jz, Fy + Fz, s11, s12);
        PAIR(13, 14, b2, ea2, ec2, kf2, kd2, uy - uz, Jy - Jz, Fy - Fz, s13, s14);
        PAIR(15, 16, b2, ea2, ec2, kf2, kd2, ux + uz, Jx + Jz, Fx + Fz, s15, s16);
        PAIR(17, 18, b2, ea2, ec2, kf2, kd2, ux - uz, Jx - Jz, Fx - Fz, s17, s18);
#undef PAIR
    }
}

// Two adjacent cells (x, x + 1), x even, per work item: for 16-bit storage
// the pair shares one 32-bit shared-memory load per population (the x shift
// of population i is taken from the pair at x for one cell and from one
// 16-bit load for the other), one packed conversion and one 32-bit store per
// population.  Each cell's arithmetic is exactly collide_group's.
template <typename S>
struct PairOf;
template <>
struct PairOf<__half> {
    using T = __half2;
    static __device__ __forceinline__ float lo(T v) { return __low2float(v); }
    static __device__ __forceinline__ float hi(T v) { return __high2float(v); }
    static __device__ __forceinline__ T pack(float a, float b) { return __floats2half2_rn(a, b); }
};
template <>
struct PairOf<__nv_bfloat16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ float lo(T v) { return __low2float(v); }
    static __device__ __forceinline__ float hi(T v) { return __high2float(v); }
    static __device__ __forceinline__ T pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

// BGK + Guo of one cell from its 19 pulled offsets s (the arithmetic of
// collide_group, for the pair path): post-collision offsets into o, the
// velocity into u.
template <bool FORCE>
__device__ __forceinline__ void bgk_guo_cell(const float (&s)[Q], float Fx, float Fy, float Fz, float omega,
                                             float rho0, float (&o)[Q], float &ux, float &uy, float &uz)
{
    const float p1 = s[1] + s[2], m1 = s[1] - s[2], p3 = s[3] + s[4], m3 = s[3] - s[4], p5 = s[5] + s[6],
                m5 = s[5] - s[6];
    const float p7 = s[7] + s[8], m7 = s[7] - s[8], p9 = s[9] + s[10], m9 = s[9] - s[10];
    const float p11 = s[11] + s[12], m11 = s[11] - s[12], p13 = s[13] + s[14], m13 = s[13] - s[14];
    const float p15 = s[15] + s[16], m15 = s[15] - s[16], p17 = s[17] + s[18], m17 = s[17] - s[18];
    const float drho = ((s[0] + p1) + (p3 + p5)) + ((p7 + p9) + (p11 + p13)) + (p15 + p17);
    const float jx = ((m1 + m7) + (m9 + m15)) + m17;
    const float jy = ((m3 + m7) - (m9 - m11)) + m13;
    const float jz = ((m5 + m11) - (m13 - m15)) - m17;
    const float rho = rho0 + drho;
    const float irho = __fdividef(1.0f, rho);
    const float Jx = FORCE ? fmaf(0.5f, Fx, jx) : jx;
    const float Jy = FORCE ? fmaf(0.5f, Fy, jy) : jy;
    const float Jz = FORCE ? fmaf(0.5f, Fz, jz) : jz;
    ux = Jx * irho;
    uy = Jy * irho;
    uz = Jz * irho;
    const float om1 = 1.0f - omega, k = fmaf(-0.5f, omega, 1.0f), er = omega * rho;
    float X = omega * fmaf(-1.5f * rho, fmaf(ux, ux, fmaf(uy, uy, uz * uz)), drho);
    if (FORCE)
        X = fmaf(-3.0f * k, fmaf(ux, Fx, fmaf(uy, Fy, uz * Fz)), X);
    o[0] = fmaf(om1, s[0], W0 * X);
    const float b1 = W1 * X, ea1 = (4.5f * W1) * er, ec1 = K1 * omega;
    const float b2 = W2 * X, ea2 = (4.5f * W2) * er, ec2 = K2 * omega;
    const float kf1 = (9.0f * W1) * k, kd1 = K1 * k, kf2 = (9.0f * W2) * k, kd2 = K2 * k;
#define PAIR(i, j, b, ea, ec, kf, kd, cu_e, cJ_e, cF_e)                                                    \
    {                                                                                                    \
        const float cu_ = (cu_e), cJ_ = (cJ_e);                                                          \
        float Pp, Mm;                                                                                    \
        if (FORCE) {                                                                                     \
            const float cF_ = (cF_e);                                                                    \
            Mm = fmaf(ec, cJ_, kd * cF_);                                                                \
            Pp = fmaf(fmaf(ea, cu_, kf * cF_), cu_, b);                                                  \
        } else {                                                                                         \
            Mm = __fmul_rn(ec, cJ_);                                                                     \
            Pp = fmaf(__fmul_rn(ea, cu_), cu_, b);                                                       \
        }                                                                                                \
        o[i] = fmaf(om1, s[i], Pp + Mm);                                                                 \
        o[j] = fmaf(om1, s[j], Pp - Mm);                                                                 \
    }
    PAIR(1, 2, b1, ea1, ec1, kf1, kd1, ux, Jx, Fx);
    PAIR(3, 4, b1, ea1, ec1, kf1, kd1, uy, Jy, Fy);
    PAIR(5, 6, b1, ea1, ec1, kf1, kd1, uz, Jz, Fz);
    PAIR(7, 8, b2, ea2, ec2, kf2, kd2, ux + uy, Jx + Jy, Fx + Fy);
    PAIR(9, 10, b2, ea2, ec2, kf2, kd2, ux - uy, Jx - Jy, Fx - Fy);
    PAIR(11, 12, b2, ea2, ec2, kf2, kd2, uy + uz, Jy + Jz, Fy + Fz);
    PAIR(13, 14, b2, ea2, ec2, kf2, kd2, uy - uz, Jy - Jz, Fy - Fz);
    PAIR(15, 16, b2, ea2, ec2, kf2, kd2, ux + uz, Jx + Jz, Fx + Fz);
    PAIR(17, 18, b2, ea2, ec2, kf2, kd2, ux - uz, Jx - Jz, Fx - Fz);
#undef PAIR
}

// omega of cell (x, y, z) of a droplet with variable tau: tau_in iff an odd
// number of the column's ray crossings lie below the cell (the in/out test)
template <bool VARTAU>
__device__ __forceinline__ float cell_omega(const Arrays &a, const DropC &c, int x, int y, int z)
{
    float omega = c.omega_out;
    if (VARTAU && c.vartau) {
        const int64_t col = c.col0 + x + (int64_t)c.nx * y;
        const int cnt = min(a.col_cnt[col], MAXC);
        const double Z = (double)(z + c.walls);
        int par = 0;
        for (int q = 0; q < cnt; ++q)
            par ^= a.col_z[col * MAXC + q] < Z;
        if (par)
            omega = c.omega_in;
    }
    return omega;
}

// kk: the block's count of groups so far.  When the group's pairs do not
// divide evenly among the consumer threads, the threads that take one pair
// more change from group to group (a rotation by kk times the remainder),
// so that no warp is always the last to release a stage.
template <typename S, bool VARTAU, bool FORCE>
__device__ __forceinline__ void collide_pairs(const Arrays &a, const DropC &c, const Stage<S> &stg, int y0, int z,
                                              int nr, bool band, S *__restrict__ dst, int kk, uint32_t gen)
{
    using PT = typename PairOf<S>::T;
    using PO = PairOf<S>;
    const int nx = c.nx, ny = c.ny, P = c.P, R = c.R;
    const int PC = c.PC;
    const int64_t pcell0 = c.pcell0;
    const bool bbm = c.walls && z == 0;            // rows pulled from z-1 bounced at the bottom
    const bool bbp = c.walls && z == c.nzf - 1;    // rows pulled from z+1 bounced at the top
    const int RP = R * P;
    S *outb = dst + (int64_t)Q * pcell0 + (int64_t)P * ny * z;
    float4 *U = a.U;
    const int npr = c.npr, step_r = c.pstep_r, step_x = c.pstep_x;
    int r = c.pr0, px = c.px0;
    constexpr int NT = cons_threads<S>();
    const int extra = (nr * npr) % NT;
    if (extra) {
        int e0 = threadIdx.x + (int)(((int64_t)kk * extra) % NT);
        if (e0 >= NT)
            e0 -= NT;
        r = e0 / npr;
        px = e0 - r * npr;
    }
    for (; r < nr; r += step_r, px += step_x) {
        if (px >= npr) {
            px -= npr;
            ++r;
            if (r >= nr)
                break;
        }
        const int x = 2 * px, y = y0 + r;
        const bool hasB = x + 1 < nx;              // an odd row ends on a single cell
        const int xm = x ? x - 1 : nx - 1;         // source of the +x populations of cell x
        const int xp2 = x + 2 < nx ? x + 2 : x + 2 - nx;   // source of the -x populations of cell x + 1
        const S *Rr = stg.pop + r * P;
        PT pv[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            pv[i] = *reinterpret_cast<const PT *>(Rr + i * RP + x);
#define SC(i, xx) cvt(Rr[(i) * RP + (xx)])
        float FAx = 0.f, FAy = 0.f, FAz = 0.f, FBx = 0.f, FBy = 0.f, FBz = 0.f;
        if (FORCE) {
            FAx = FBx = c.bfx;
            FAy = FBy = c.bfy;
            FAz = FBz = c.bfz;
            if (band) {     // F vanishes outside band tiles
                const float *Fr = stg.F + r * P + x;
                const float2 f0 = *reinterpret_cast<const float2 *>(Fr);
                const float2 f1 = *reinterpret_cast<const float2 *>(Fr + RP);
                const float2 f2 = *reinterpret_cast<const float2 *>(Fr + 2 * RP);
                FAx += f0.x;
                FBx += f0.y;
                FAy += f1.x;
                FBy += f1.y;
                FAz += f2.x;
                FBz += f2.y;
            }
        }
        const int64_t cell = (int64_t)P * (y + (int64_t)ny * z) + x;
        S *o = outb + P * y + x;
        const bool ub = FORCE && band && in_band_tile(a, c, x, y, z, gen);   // both cells share the tile
        float oa[Q];
        {   // cell x: c_x = 0 from the pair's low half, +x from x - 1, -x from the pair's high half
            float sa[Q];
            sa[0] = PO::lo(pv[0]);
            sa[3] = PO::lo(pv[3]);
            sa[4] = PO::lo(pv[4]);
            sa[5] = PO::lo(pv[5]);
            sa[6] = PO::lo(pv[6]);
            sa[11] = PO::lo(pv[11]);
            sa[12] = PO::lo(pv[12]);
            sa[13] = PO::lo(pv[13]);
            sa[14] = PO::lo(pv[14]);
            sa[1] = SC(1, xm);
            sa[7] = SC(7, xm);
            sa[9] = SC(9, xm);
            sa[15] = bbm ? PO::lo(pv[15]) : SC(15, xm);
            sa[17] = bbp ? PO::lo(pv[17]) : SC(17, xm);
            // (the -x populations of the last cell of an odd row wrap to x = 0)
            sa[2] = hasB ? PO::hi(pv[2]) : SC(2, 0);
            sa[8] = hasB ? PO::hi(pv[8]) : SC(8, 0);
            sa[10] = hasB ? PO::hi(pv[10]) : SC(10, 0);
            sa[16] = bbp ? PO::lo(pv[16]) : (hasB ? PO::hi(pv[16]) : SC(16, 0));
            sa[18] = bbm ? PO::lo(pv[18]) : (hasB ? PO::hi(pv[18]) : SC(18, 0));
            float ux, uy, uz;
            bgk_guo_cell<FORCE>(sa, FAx, FAy, FAz, cell_omega<VARTAU>(a, c, x, y, z), c.rho0, oa, ux, uy, uz);
            if (FORCE && ub) {
                const int64_t gi = pcell0 + cell;
                U[gi] = make_float4(ux, uy, uz, 0.0f);
            }
        }
        if (hasB) {  // cell x + 1: c_x = 0 from the high half, +x from the low half, -x from x + 2
            float sb[Q], ob[Q];
            sb[0] = PO::hi(pv[0]);
            sb[3] = PO::hi(pv[3]);
            sb[4] = PO::hi(pv[4]);
            sb[5] = PO::hi(pv[5]);
            sb[6] = PO::hi(pv[6]);
            sb[11] = PO::hi(pv[11]);
            sb[12] = PO::hi(pv[12]);
            sb[13] = PO::hi(pv[13]);
            sb[14] = PO::hi(pv[14]);
            sb[1] = PO::lo(pv[1]);
            sb[7] = PO::lo(pv[7]);
            sb[9] = PO::lo(pv[9]);
            sb[15] = bbm ? PO::hi(pv[15]) : PO::lo(pv[15]);
            sb[17] = bbp ? PO::hi(pv[17]) : PO::lo(pv[17]);
            sb[2] = SC(2, xp2);
            sb[8] = SC(8, xp2);
            sb[10] = SC(10, xp2);
            sb[16] = bbp ? PO::hi(pv[16]) : SC(16, xp2);
            sb[18] = bbm ? PO::hi(pv[18]) : SC(18, xp2);
            float ux, uy, uz;
            bgk_guo_cell<FORCE>(sb, FBx, FBy, FBz, cell_omega<VARTAU>(a, c, x + 1, y, z), c.rho0, ob, ux, uy, uz);
            if (FORCE && ub) {
                const int64_t gi = pcell0 + cell + 1;
                U[gi] = make_float4(ux, uy, uz, 0.0f);
            }
#pragma unroll
            for (int i = 0; i < Q; ++i)
                __stcs(reinterpret_cast<PT *>(o + (int64_t)i * PC), PO::pack(oa[i], ob[i]));
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                st(o + (int64_t)i * PC, oa[i]);
        }
#undef SC
    }
}

template <typename S, bool VARTAU, bool TR>
__global__ void __launch_bounds__(lb_block<S>(), 2)
    lb_kernel(Arrays a, const S *__restrict__ src, S *__restrict__ dst, int ns, const int *__restrict__ list,
              const int *__restrict__ count, int no_force, unsigned long long *tr)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // full[s]: the stage's bulk copies landed (32 producer lanes arrive with
    // the byte count); empty[s]: every consumer thread is done reading it
    __shared__ __align__(8) uint64_t full[LB_MAX_STAGES], empty[LB_MAX_STAGES];
    griddep_wait();
    if constexpr (TR)
        lb_trace_start(tr);
    const uint32_t gen = *a.gen;
    // the groups of this launch: list[0 .. *count) or all of them
    const int total = list ? *count : a.lb_blocks_total;
    if (threadIdx.x == 0) {
        for (int i = 0; i < ns; ++i) {
            mbar_init(&full[i], 32);
            mbar_init(&empty[i], cons_threads<S>());
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // Group k of this block (ig = blockIdx.x + k gridDim.x) goes through
    // stage k mod ns, whose (k / ns)-th use it is.  The producer refills a
    // stage as soon as the consumers released its previous use, so up to ns
    // groups are in flight; each consumer warp moves on to the next group as
    // soon as its data landed, without waiting for the other warps.
    bool failed = false;
    if (threadIdx.x >= cons_threads<S>()) {
        int st_i = 0;
        uint32_t use = 0, bits = 0;
        DropC c;
        c.d = -1;
        for (int ig = blockIdx.x, k = 0; ig < total; ig += gridDim.x, ++k) {
            // the band flags of the next 32 groups at once: one round trip
            // to memory per 32 groups, off the path of each group's copies
            if ((k & 31) == 0)
                bits = no_force ? 0u : band_ballot(a, list, total, ig, gridDim.x, gen);
            if (use > 0 && !mbar_wait_bounded(&empty[st_i], (use - 1) & 1u, WAIT_CYCLES)) {
                failed = true;
                break;
            }
            // order the consumers' generic reads of the stage before the
            // asynchronous writes into it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int g = list ? list[ig] : ig;
            const int d = find_drop_group(a.drops, a.ndrops, g);
            if (d != c.d)
                c.load(a.drops[d], d, cons_threads<S>());
            int y0, z, nr;
            c.rows(g, y0, z, nr);
            produce<S>(a, c, src, y0, z, nr, smem_raw + st_i * a.lb_stage_bytes, &full[st_i],
                       ((bits >> (k & 31)) & 1u) != 0);
            if (++st_i == ns) {
                st_i = 0;
                ++use;
            }
        }
    } else {
        int st_i = 0, kk = 0;
        uint32_t phase = 0;
        DropC c;
        c.d = -1;
        for (int ig = blockIdx.x; ig < total; ig += gridDim.x, ++kk) {
            const int g = list ? list[ig] : ig;
            const int d = find_drop_group(a.drops, a.ndrops, g);
            if (d != c.d)
                c.load(a.drops[d], d, cons_threads<S>());
            int y0, z, nr;
            c.rows(g, y0, z, nr);
            if (!mbar_wait_bounded(&full[st_i], phase, WAIT_CYCLES)) {
                failed = true;
                break;
            }
            const Stage<S> stg(smem_raw + st_i * a.lb_stage_bytes, c.R, c.P);
            const bool band = *stg.flag != 0;
            if constexpr (sizeof(S) == 2) {      // 16-bit storage: two cells per work item
                if (band || c.has_bf)
                    collide_pairs<S, VARTAU, true>(a, c, stg, y0, z, nr, band, dst, kk, gen);
                else
                    collide_pairs<S, VARTAU, false>(a, c, stg, y0, z, nr, false, dst, kk, gen);
            } else {
                if (band || c.has_bf)
                    collide_group<S, VARTAU, true>(a, c, stg, y0, z, nr, band, dst, gen);
                else
                    collide_group<S, VARTAU, false>(a, c, stg, y0, z, nr, false, dst, gen);
            }
            mbar_arrive(&empty[st_i]);
            if (++st_i == ns) {
                st_i = 0;
                phase ^= 1u;
            }
        }
    }
    // a bounded wait gave up: flag it and leave (a thread that leaves early
    // makes the waits of the others on it give up in turn)
    if (failed)
        atomicOr(&a.status[0], ST_TIMEOUT);
}
template <typename S>
cudaError_t launch_t(const Arrays &a, const void *src, void *dst, bool vartau, const LaunchCfg &cfg,
                     cudaStream_t s, const int *list, const int *count, bool no_force, int blocks_per_sm)
{
    const int total = a.lb_blocks_total;      // at most this many groups in a list
    if (total <= 0)
        return cudaSuccess;
    const int ns = cfg.lb_stages < 2 ? 2 : (cfg.lb_stages > LB_MAX_STAGES ? LB_MAX_STAGES : cfg.lb_stages);
    const size_t smem = (size_t)ns * a.lb_stage_bytes;
    const bool traced = g_trace_lb != nullptr;
    const void *fn = vartau ? (traced ? (const void *)lb_kernel<S, true, true> : (const void *)lb_kernel<S, true, false>)
                            : (traced ? (const void *)lb_kernel<S, false, true> : (const void *)lb_kernel<S, false, false>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, lb_block<S>(), smem);
    if (e != cudaSuccess)
        return e;
    if (per_sm < 1)
        return cudaErrorInvalidConfiguration;
    const int want = blocks_per_sm >= 0 ? blocks_per_sm : cfg.lb_blocks_per_sm;
    if (want > 0 && want < per_sm)
        per_sm = want;
    int grid = cfg.sm_count * per_sm;
    grid = grid < total ? grid : total;
    const int nf = no_force ? 1 : 0;
    unsigned long long *tr = g_trace_lb;
    const dim3 g(grid), b(lb_block<S>());
    if (vartau)
        return traced ? launch_k(lb_kernel<S, true, true>, g, b, smem, s, a.pdl != 0, a, (const S *)src, (S *)dst, ns,
                                 list, count, nf, tr)
                      : launch_k(lb_kernel<S, true, false>, g, b, smem, s, a.pdl != 0, a, (const S *)src, (S *)dst, ns,
                                 list, count, nf, tr);
    return traced ? launch_k(lb_kernel<S, false, true>, g, b, smem, s, a.pdl != 0, a, (const S *)src, (S *)dst, ns, list,
                             count, nf, tr)
                  : launch_k(lb_kernel<S, false, false>, g, b, smem, s, a.pdl != 0, a, (const S *)src, (S *)dst, ns,
                             list, count, nf, tr);
}

}  // namespace

int lb_rows_per_group(int nx) { return nx >= LB_THREADS ? 1 : LB_THREADS / nx; }

int lb_stage_bytes(int rows, int pitch, int sb)
{
    const size_t b = (size_t)rows * Q * pitch * sb + (size_t)rows * 3 * pitch * sizeof(float) + 16;
    return (int)((b + 127) & ~(size_t)127);
}

cudaError_t launch_lb(const Arrays &a, int storage, const void *src, void *dst, bool vartau,
                      const LaunchCfg &cfg, cudaStream_t s, const int *list, const int *count, bool no_force,
                      int blocks_per_sm)
{
    switch (storage) {
    case 0: return launch_t<float>(a, src, dst, vartau, cfg, s, list, count, no_force, blocks_per_sm);
    case 1: return launch_t<__half>(a, src, dst, vartau, cfg, s, list, count, no_force, blocks_per_sm);
    case 2: return launch_t<__nv_bfloat16>(a, src, dst, vartau, cfg, s, list, count, no_force, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
}

namespace {

__device__ __forceinline__ int find_drop_trow(const Drop *D, int n, int64_t r)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].trow0 <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Did the previous step (generation gprev) put a tile into a tile row within
// one row of rows ty0 .. ty1 (y wraps) and tz (z wraps without walls)?
__device__ bool near_band(const Arrays &a, const Drop &D, int ty0, int ty1, int tz, uint32_t gprev)
{
    for (int dz = -1; dz <= 1; ++dz) {
        int zz = tz + dz;
        if (D.walls) {
            if (zz < 0 || zz >= D.tz)
                continue;
        } else {
            zz = wrapi(zz, D.tz);
        }
        const int ny = ty1 - ty0 + 3 < D.ty ? ty1 - ty0 + 3 : D.ty;
        for (int k = 0; k < ny; ++k) {
            const int yy = ny == D.ty ? k : wrapi(ty0 - 1 + k, D.ty);
            if (a.rowgen[D.trow0 + yy + (int64_t)D.ty * zz] == gprev)
                return true;
        }
    }
    return false;
}

// One thread per tile row, then one per stream-collide group.  A node moves
// less than half a cell per step (faster nodes stop the run with an error),
// so a tile of the coming step's band lies within one tile of a tile of the
// previous band: its tile row is within one row of a row that held band
// tiles.  The groups that cross no such row carry no force in the coming
// step and can run before its forces are known.  Without a previous band
// (*split_ok == 0) every row and group counts as near.
__global__ void __launch_bounds__(256) classify_kernel(Arrays a)
{
    const uint32_t gprev = *a.gen;
    const bool ok = *a.split_ok != 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid == 0)
        a.grp_cnt[2] = 1;             // the force kernel checks this step's band against candrow
    for (int64_t r = gid; r < a.total_trows; r += stride) {
        const Drop &D = a.drops[find_drop_trow(a.drops, a.ndrops, r)];
        const int local = (int)(r - D.trow0);
        const int ty = local % D.ty, tz = local / D.ty;
        a.candrow[r] = (!ok || near_band(a, D, ty, ty, tz, gprev)) ? 1 : 0;
    }
    for (int64_t g = gid; g < a.lb_blocks_total; g += stride) {
        const Drop &D = a.drops[find_drop_group(a.drops, a.ndrops, (int)g)];
        int y0, z, nr;
        group_rows(D, (int)g, y0, z, nr);
        const bool near = !ok || near_band(a, D, y0 >> 2, (y0 + nr - 1) >> 2, z >> 2, gprev);
        const int slot = atomicAdd(&a.grp_cnt[near ? 0 : 1], 1);
        a.grp_list[(near ? 0 : a.total_rows) + slot] = (int)g;
    }
}

}  // namespace

void set_trace_lb(unsigned long long *trace) { g_trace_lb = trace; }

cudaError_t launch_classify(const Arrays &a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.grp_cnt, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    const int64_t n = a.total_trows > a.lb_blocks_total ? a.total_trows : a.lb_blocks_total;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    classify_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace iblb
