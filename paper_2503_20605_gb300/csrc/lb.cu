// lb.cu -- fused pull-stream + halfway bounce-back + moments + BGK + Guo
// source for D3Q19 (Sec. II A: eqs. LBE, hydro_var1, hydro_var2, the BGK
// operator, the equilibrium and Guo's source term), one lattice cell per
// thread, populations stored as offsets s_i = f_i - w_i rho0 in FP32, FP16
// or BF16 with all arithmetic in FP32.
//
// Memory traffic per fluid cell: 19 loads and 19 stores of the storage type
// (152 B for FP32, 76 B for 16-bit storage).  The force density is read and
// the velocity written only on cells of the band tiles around the membrane.
#include "iblb_internal.h"

namespace iblb {

namespace {

__device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ void st(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st(__half *p, float v) { __stcs(reinterpret_cast<unsigned short *>(p), __half_as_ushort(__float2half_rn(v))); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { __stcs(reinterpret_cast<unsigned short *>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v))); }

__device__ __forceinline__ int find_drop_block(const Drop *D, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].lb_block0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

constexpr float W0 = 1.0f / 3.0f, W1 = 1.0f / 18.0f, W2 = 1.0f / 36.0f;

template <typename S, bool VARTAU>
__global__ void __launch_bounds__(512) lb_kernel(Arrays a, const S *__restrict__ src, S *__restrict__ dst)
{
    const uint32_t gen = *a.gen;
    for (int b = blockIdx.x; b < a.lb_blocks_total; b += gridDim.x) {
        const int d = find_drop_block(a.drops, a.ndrops, b);
        const Drop &D = a.drops[d];
        const int nx = D.nx, ny = D.ny, nzf = D.nzf;
        const int64_t N = D.cells;
        const int64_t c = (int64_t)(b - D.lb_block0) * a.lb_cpb + threadIdx.x;
        if (c >= N)
            continue;
        const int ci = (int)c;
        const int x = ci % nx;
        const int yz = ci / nx;
        const int y = yz % ny;
        const int z = yz / ny;
        const int xm = x ? x - 1 : nx - 1, xp = x + 1 < nx ? x + 1 : 0;
        const int ym = y ? y - 1 : ny - 1, yp = y + 1 < ny ? y + 1 : 0;
        const bool zlo = z == 0, zhi = z == nzf - 1;
        const bool bbm = D.walls && zlo;   // pulling from z-1 reaches the bottom wall
        const bool bbp = D.walls && zhi;   // pulling from z+1 reaches the top wall
        const int zm = zlo ? (D.walls ? 0 : nzf - 1) : z - 1;
        const int zp = zhi ? (D.walls ? 0 : 0) : z + 1;
        const int r00 = nx * (y + ny * z), rm0 = nx * (ym + ny * z), rp0 = nx * (yp + ny * z);
        const int r0m = nx * (y + ny * zm), r0p = nx * (y + ny * zp);
        const int rmm = nx * (ym + ny * zm), rpm = nx * (yp + ny * zm);
        const int rmp = nx * (ym + ny * zp), rpp = nx * (yp + ny * zp);

        const S *f = src + (int64_t)Q * D.cell0;
#define P(i) (f + (int64_t)(i) * N)
        // pull: s_i(x) = s*_i(x - c_i); halfway bounce-back at a resting wall
        const float s0 = ld(P(0) + x + r00);
        const float s1 = ld(P(1) + xm + r00);
        const float s2 = ld(P(2) + xp + r00);
        const float s3 = ld(P(3) + x + rm0);
        const float s4 = ld(P(4) + x + rp0);
        const float s5 = bbm ? ld(P(6) + ci) : ld(P(5) + x + r0m);
        const float s6 = bbp ? ld(P(5) + ci) : ld(P(6) + x + r0p);
        const float s7 = ld(P(7) + xm + rm0);
        const float s8 = ld(P(8) + xp + rp0);
        const float s9 = ld(P(9) + xm + rp0);
        const float s10 = ld(P(10) + xp + rm0);
        const float s11 = bbm ? ld(P(12) + ci) : ld(P(11) + x + rmm);
        const float s12 = bbp ? ld(P(11) + ci) : ld(P(12) + x + rpp);
        const float s13 = bbp ? ld(P(14) + ci) : ld(P(13) + x + rmp);
        const float s14 = bbm ? ld(P(13) + ci) : ld(P(14) + x + rpm);
        const float s15 = bbm ? ld(P(16) + ci) : ld(P(15) + xm + r0m);
        const float s16 = bbp ? ld(P(15) + ci) : ld(P(16) + xp + r0p);
        const float s17 = bbp ? ld(P(18) + ci) : ld(P(17) + xm + r0p);
        const float s18 = bbm ? ld(P(17) + ci) : ld(P(18) + xp + r0m);
#undef P

        // force density: band tiles carry the spread IB force
        float Fx = D.bf[0], Fy = D.bf[1], Fz = D.bf[2];
        const int64_t gcell = D.cell0 + c;
        const int64_t tile = D.tile0 + (x >> 2) + (int64_t)D.tx * ((y >> 2) + (int64_t)D.ty * (z >> 2));
        const bool band = a.tile_gen[tile] == gen;
        if (band) {
            Fx += a.F[gcell];
            Fy += a.F[a.total_cells + gcell];
            Fz += a.F[2 * a.total_cells + gcell];
        }

        float omega = D.omega_out;
        if (VARTAU && D.vartau) {
            const int64_t col = D.col0 + x + (int64_t)nx * y;
            const int cnt = min(a.col_cnt[col], MAXC);
            const double Z = (double)(z + D.walls);
            int par = 0;
            for (int k = 0; k < cnt; ++k)
                par ^= a.col_z[col * MAXC + k] < Z;
            if (par)
                omega = D.omega_in;
        }

        // moments (eqs. hydro_var1, hydro_var2) in offset form
        const float drho = ((s0 + (s1 + s2)) + ((s3 + s4) + (s5 + s6))) +
                           (((s7 + s8) + (s9 + s10)) + ((s11 + s12) + (s13 + s14))) +
                           ((s15 + s16) + (s17 + s18));
        const float jx = (s1 - s2) + (s7 - s8) + (s9 - s10) + (s15 - s16) + (s17 - s18);
        const float jy = (s3 - s4) + (s7 - s8) - (s9 - s10) + (s11 - s12) + (s13 - s14);
        const float jz = (s5 - s6) + (s11 - s12) - (s13 - s14) + (s15 - s16) - (s17 - s18);
        const float rho = D.rho0 + drho;
        const float irho = 1.0f / rho;
        const float ux = (jx + 0.5f * Fx) * irho;
        const float uy = (jy + 0.5f * Fy) * irho;
        const float uz = (jz + 0.5f * Fz) * irho;
        if (band) {
            a.U[gcell] = ux;
            a.U[a.total_cells + gcell] = uy;
            a.U[2 * a.total_cells + gcell] = uz;
        }

        // BGK + Guo: s*_i = s_i + omega (s_eq_i - s_i) + S_i with
        // s_eq_i = w_i [drho + rho (3 cu + 9/2 cu^2 - 3/2 u.u)]  (f_eq - w_i rho0)
        // S_i    = (1 - omega/2) w_i [3 (c_i - U).F + 9 (c_i.U)(c_i.F)]
        const float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
        const float uF3 = 3.0f * (ux * Fx + uy * Fy + uz * Fz);
        const float kS = 1.0f - 0.5f * omega;
        S *o = dst + (int64_t)Q * D.cell0 + c;
#define COLL(i, w, cu, cF, si)                                                              \
    {                                                                                        \
        const float cu_ = (cu), cF_ = (cF);                                                  \
        const float seq = (w) * (drho + rho * (3.0f * cu_ + 4.5f * cu_ * cu_ - uu15));       \
        const float Si = kS * (w) * (3.0f * cF_ - uF3 + 9.0f * cu_ * cF_);                   \
        st(o + (int64_t)(i) * N, (si) + omega * (seq - (si)) + Si);                          \
    }
        COLL(0, W0, 0.0f, 0.0f, s0);
        COLL(1, W1, ux, Fx, s1);
        COLL(2, W1, -ux, -Fx, s2);
        COLL(3, W1, uy, Fy, s3);
        COLL(4, W1, -uy, -Fy, s4);
        COLL(5, W1, uz, Fz, s5);
        COLL(6, W1, -uz, -Fz, s6);
        COLL(7, W2, ux + uy, Fx + Fy, s7);
        COLL(8, W2, -ux - uy, -Fx - Fy, s8);
        COLL(9, W2, ux - uy, Fx - Fy, s9);
        COLL(10, W2, -ux + uy, -Fx + Fy, s10);
        COLL(11, W2, uy + uz, Fy + Fz, s11);
        COLL(12, W2, -uy - uz, -Fy - Fz, s12);
        COLL(13, W2, uy - uz, Fy - Fz, s13);
        COLL(14, W2, -uy + uz, -Fy + Fz, s14);
        COLL(15, W2, ux + uz, Fx + Fz, s15);
        COLL(16, W2, -ux - uz, -Fx - Fz, s16);
        COLL(17, W2, ux - uz, Fx - Fz, s17);
        COLL(18, W2, -ux + uz, -Fx + Fz, s18);
#undef COLL
    }
}

template <typename S>
cudaError_t launch_t(const Arrays &a, const void *src, void *dst, bool vartau, const LaunchCfg &cfg,
                     cudaStream_t s)
{
    int grid = a.lb_blocks_total;
    if (grid <= 0)
        return cudaSuccess;
    if (cfg.lb_persistent) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, vartau ? (const void *)lb_kernel<S, true> : (const void *)lb_kernel<S, false>,
            cfg.lb_block, 0);
        int g = cfg.sm_count * (per_sm > 0 ? per_sm : 1);
        grid = grid < g ? grid : g;
    }
    if (vartau)
        lb_kernel<S, true><<<grid, cfg.lb_block, 0, s>>>(a, (const S *)src, (S *)dst);
    else
        lb_kernel<S, false><<<grid, cfg.lb_block, 0, s>>>(a, (const S *)src, (S *)dst);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lb(const Arrays &a, int storage, const void *src, void *dst, bool vartau,
                      const LaunchCfg &cfg, cudaStream_t s)
{
    switch (storage) {
    case 0: return launch_t<float>(a, src, dst, vartau, cfg, s);
    case 1: return launch_t<__half>(a, src, dst, vartau, cfg, s);
    case 2: return launch_t<__nv_bfloat16>(a, src, dst, vartau, cfg, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace iblb
