// ib.cu -- the membrane side of the IB-LB step:
//   * nodal forces: surface tension phi_sigma,j = -sigma dA/dq_j (Sec. II B)
//     plus the wall interaction phi_Pi,j = -(chi_j/3) Pi(h_j) n_j (Sec. II C),
//     one thread per node gathering over its incident faces in a fixed order;
//   * force spreading F(x) = sum_j phi_j Delta(q_j - x) (eq. force_spread) as
//     a deterministic binned gather: nodes are binned by the 4^3 tile of their
//     support's base cell, every band tile gathers the nodes overlapping it
//     and adds their contributions in increasing node index, so the result
//     does not depend on launch shapes or on the other droplets of a batch;
//   * interpolation qdot_j = sum_x U(x) Delta(q_j - x) (eq. vel_interpolation)
//     and forward-Euler advection q_j += qdot_j, 16 lanes per node.
// Node positions are FP64 so that edge vectors and kernel offsets are exact
// before they are rounded to FP32 for the force and kernel arithmetic.
#include "iblb_internal.h"

namespace iblb {

namespace {

__device__ __forceinline__ float psi_near(float r)  // 0 <= r <= 1
{
    return 0.375f - 0.25f * r + 0.25f * sqrtf(r - r * r + 0.25f);
}
__device__ __forceinline__ float psi_far(float r)   // 1 <= r <= 2
{
    return 0.625f - 0.25f * r - 0.25f * sqrtf(3.0f * r - r * r - 1.75f);
}

__device__ __forceinline__ float ipow(float r, int k)
{
    float p = 1.0f;
    for (int i = 0; i < k; ++i)
        p *= r;
    return p;
}

__device__ __forceinline__ int tile_key(const Drop &D, int bx, int by, int bz)
{
    // base cell in fluid coordinates (x, y wrapped); -1 if the support misses the fluid
    int tz;
    if (D.walls) {
        if (bz + 2 < 0 || bz - 1 >= D.nzf)
            return -1;
        tz = floordiv(bz, TILE);
        tz = tz < 0 ? 0 : (tz >= D.tz ? D.tz - 1 : tz);
    } else {
        tz = bz >> 2;
    }
    return (bx >> 2) + D.tx * ((by >> 2) + D.ty * tz);
}

// One thread per node.  Thread 0 also opens the step: generation += 1 and an
// empty band list.
__global__ void node_force_kernel(Arrays a)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {
        *a.gen += 1u;
        *a.n_active = 0;
    }
    if (j >= a.total_nodes)
        return;
    const int d = a.node_drop[j];
    const Drop &D = a.drops[d];
    const double qx = a.qx[j], qy = a.qy[j], qz = a.qz[j];
    float gx = 0.f, gy = 0.f, gz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f, chi = 0.f;
    for (int e = a.adj_start[j]; e < a.adj_start[j + 1]; ++e) {
        const int code = a.adj[e];
        const int t = code >> 2, k = code & 3;
        const int v0 = a.tri[3 * t], v1 = a.tri[3 * t + 1], v2 = a.tri[3 * t + 2];
        const double x0 = a.qx[v0], y0 = a.qy[v0], z0 = a.qz[v0];
        const float e1x = (float)(a.qx[v1] - x0), e1y = (float)(a.qy[v1] - y0), e1z = (float)(a.qz[v1] - z0);
        const float e2x = (float)(a.qx[v2] - x0), e2y = (float)(a.qy[v2] - y0), e2z = (float)(a.qz[v2] - z0);
        const float Nx = e1y * e2z - e1z * e2y;
        const float Ny = e1z * e2x - e1x * e2z;
        const float Nz = e1x * e2y - e1y * e2x;
        const float len = sqrtf(Nx * Nx + Ny * Ny + Nz * Nz);
        const float il = 1.0f / len;
        const float hx = Nx * il, hy = Ny * il, hz = Nz * il;
        // dA/dq_k = 1/2 n x (q_prev - q_next), corners in CCW order
        const int vp = k == 0 ? v2 : (k == 1 ? v0 : v1);
        const int vn = k == 0 ? v1 : (k == 1 ? v2 : v0);
        const float dx = (float)(a.qx[vp] - a.qx[vn]);
        const float dy = (float)(a.qy[vp] - a.qy[vn]);
        const float dz = (float)(a.qz[vp] - a.qz[vn]);
        gx += 0.5f * (hy * dz - hz * dy);
        gy += 0.5f * (hz * dx - hx * dz);
        gz += 0.5f * (hx * dy - hy * dx);
        nx += hx;
        ny += hy;
        nz += hz;
        chi += 0.5f * len;
    }
    float px = -D.sigma * gx, py = -D.sigma * gy, pz = -D.sigma * gz;
    if (D.wetting) {
        float h = (float)(qz - 0.5);
        if (h < D.hmin) {
            h = D.hmin;
            atomicAdd(&a.clamped[d], 1);
        }
        const float r = D.xi / h;
        const float Pi = D.A * (ipow(r, D.n) - ipow(r, D.m));
        const float inl = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
        const float s = -(chi * (1.0f / 3.0f)) * Pi * inl;
        px += s * nx;
        py += s * ny;
        pz += s * nz;
    }
    NodeRec r;
    if (!(fabs(qx) < 1e8 && fabs(qy) < 1e8 && fabs(qz) < 1e8)) {
        // non-finite or absurd position: no support, no bin, flagged
        atomicOr(&a.status[4 * d], ST_NAN);
        r.bx = r.by = r.bz = 0;
        r.key = -1;
        for (int k = 0; k < 4; ++k)
            r.wx[k] = r.wy[k] = r.wz[k] = 0.0f;
        r.phi[0] = r.phi[1] = r.phi[2] = 0.0f;
        r.spare = 0;
        a.rec[j] = r;
        return;
    }
    // support of the 4-point kernel: base-1 .. base+2 on each axis
    const double fbx = floor(qx), fby = floor(qy), fbz = floor(qz);
    const float fx = (float)(qx - fbx), fy = (float)(qy - fby), fz = (float)(qz - fbz);
    r.bx = wrapi((int)fbx % D.nx, D.nx);
    r.by = wrapi((int)fby % D.ny, D.ny);
    int bz = (int)fbz - D.walls;
    if (!D.walls)
        bz = wrapi(bz % D.nz, D.nz);
    r.bz = bz;
    r.wx[0] = psi_far(1.0f + fx); r.wx[1] = psi_near(fx); r.wx[2] = psi_near(1.0f - fx); r.wx[3] = psi_far(2.0f - fx);
    r.wy[0] = psi_far(1.0f + fy); r.wy[1] = psi_near(fy); r.wy[2] = psi_near(1.0f - fy); r.wy[3] = psi_far(2.0f - fy);
    r.wz[0] = psi_far(1.0f + fz); r.wz[1] = psi_near(fz); r.wz[2] = psi_near(1.0f - fz); r.wz[3] = psi_far(2.0f - fz);
    r.phi[0] = px;
    r.phi[1] = py;
    r.phi[2] = pz;
    r.spare = 0;
    const int key = tile_key(D, r.bx, r.by, r.bz);
    r.key = key < 0 ? -1 : (int)(D.tile0 + key);
    if (key < 0)
        atomicOr(&a.status[4 * d], ST_ESCAPE);
    else
        atomicAdd(&a.bin_cnt[r.key], 1);
    a.rec[j] = r;
}

// Block-level exclusive scan of the bin counts (SCAN_ITEMS per block).
__global__ void __launch_bounds__(1024) scan_blocks_kernel(const int *__restrict__ cnt, int64_t n,
                                                           int *__restrict__ off, int *__restrict__ blk_sum)
{
    __shared__ int warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS + 4 * threadIdx.x;
    int v[4];
    for (int i = 0; i < 4; ++i)
        v[i] = base + i < n ? cnt[base + i] : 0;
    const int local = v[0] + v[1] + v[2] + v[3];
    int inc = local;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += t;
    }
    if (lane == 31)
        warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < (blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int run = inc - local + (w ? warp_tot[w - 1] : 0);
    for (int i = 0; i < 4; ++i) {
        if (base + i < n)
            off[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == blockDim.x - 1)
        blk_sum[blockIdx.x] = warp_tot[(blockDim.x >> 5) - 1];
}

// Exclusive scan of the block totals by one block (serial over chunks of 1024).
__global__ void __launch_bounds__(1024) scan_top_kernel(const int *__restrict__ blk_sum, int nb,
                                                        int *__restrict__ blk_off)
{
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        const int v = i < nb ? blk_sum[i] : 0;
        int inc = v;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += t;
        }
        if (lane == 31)
            warp_tot[w] = inc;
        __syncthreads();
        if (w == 0) {
            int t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o)
                    t += u;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int ex = inc - v + (w ? warp_tot[w - 1] : 0) + carry;
        if (i < nb)
            blk_off[i] = ex;
        __syncthreads();
        if (threadIdx.x == 1023)
            carry = ex + v;
        __syncthreads();
    }
}

// start of bin t in bin_list; the scan covers total_tiles + 1 entries (the
// last count is always zero), so bin t ends where bin t + 1 begins
__device__ __forceinline__ int bin_begin(const Arrays &a, int64_t t)
{
    return a.bin_off[t] + a.blk_off[t / SCAN_ITEMS];
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

// Place every binned node in its bin (order inside a bin is irrelevant: the
// gather sorts by node index).  The node that empties its bin counter marks
// the tiles around the bin as band tiles of this step.
__global__ void fill_kernel(Arrays a)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.total_nodes)
        return;
    const int key = a.rec[j].key;
    if (key < 0)
        return;
    const int old = atomicSub(&a.bin_cnt[key], 1);
    a.bin_list[bin_begin(a, key) + old - 1] = j;
    if (old != 1)
        return;
    const uint32_t gen = *a.gen;
    const int d = find_drop_tile(a.drops, a.ndrops, key);
    const Drop &D = a.drops[d];
    const int local = key - (int)D.tile0;
    const int kx = local % D.tx, ky = (local / D.tx) % D.ty, kz = local / (D.tx * D.ty);
    int lx[4], ly[4], lz[4];
    const int nxl = tile_neighbours(kx, D.tx, D.nx, true, lx);
    const int nyl = tile_neighbours(ky, D.ty, D.ny, true, ly);
    const int nzl = tile_neighbours(kz, D.tz, D.nzf, !D.walls, lz);
    for (int iz = 0; iz < nzl; ++iz)
        for (int iy = 0; iy < nyl; ++iy)
            for (int ix = 0; ix < nxl; ++ix) {
                const int64_t t = D.tile0 + lx[ix] + (int64_t)D.tx * (ly[iy] + (int64_t)D.ty * lz[iz]);
                if (atomicExch(&a.tile_gen[t], gen) != gen) {
                    const int s = atomicAdd(a.n_active, 1);
                    if (s < a.active_cap)
                        a.active[s] = (int)t;
                }
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

__device__ __forceinline__ bool support_hits(int lo, int hi, int b, int n, bool periodic)
{
    for (int X = lo; X <= hi; ++X) {
        const int d = periodic ? per_off(X, b, n) : X - b;
        if (d >= -1 && d <= 2)
            return true;
    }
    return false;
}

// One 64-thread block per band tile (block-stride over the band list); each
// thread owns one cell of the tile.
__global__ void __launch_bounds__(TILE_CELLS) spread_kernel(Arrays a)
{
    __shared__ int s_cnt;
    __shared__ int s_node[SPREAD_CAP];
    __shared__ short s_perm[SPREAD_CAP];
    __shared__ int s_b[3][SPREAD_CAP];
    __shared__ float s_w[12][SPREAD_CAP];
    __shared__ float s_phi[3][SPREAD_CAP];
    const int nact = min(*a.n_active, a.active_cap);
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < nact; it += gridDim.x) {
        const int64_t T = a.active[it];
        const int d = find_drop_tile(a.drops, a.ndrops, T);
        const Drop &D = a.drops[d];
        const int local = (int)(T - D.tile0);
        const int kx = local % D.tx, ky = (local / D.tx) % D.ty, kz = local / (D.tx * D.ty);
        const int X0 = 4 * kx, Y0 = 4 * ky, Z0 = 4 * kz;
        const int X1 = min(X0 + 3, D.nx - 1), Y1 = min(Y0 + 3, D.ny - 1), Z1 = min(Z0 + 3, D.nzf - 1);
        int lx[4], ly[4], lz[4];
        const int nxl = tile_neighbours(kx, D.tx, D.nx, true, lx);
        const int nyl = tile_neighbours(ky, D.ty, D.ny, true, ly);
        const int nzl = tile_neighbours(kz, D.tz, D.nzf, !D.walls, lz);
        if (tid == 0)
            s_cnt = 0;
        __syncthreads();
        for (int iz = 0; iz < nzl; ++iz)
            for (int iy = 0; iy < nyl; ++iy)
                for (int ix = 0; ix < nxl; ++ix) {
                    const int64_t B = D.tile0 + lx[ix] + (int64_t)D.tx * (ly[iy] + (int64_t)D.ty * lz[iz]);
                    const int e0 = bin_begin(a, B), e1 = bin_begin(a, B + 1);
                    for (int e = e0 + tid; e < e1; e += TILE_CELLS) {
                        const int j = a.bin_list[e];
                        const NodeRec &r = a.rec[j];
                        if (!support_hits(X0, X1, r.bx, D.nx, true) || !support_hits(Y0, Y1, r.by, D.ny, true) ||
                            !support_hits(Z0, Z1, r.bz, D.nzf, !D.walls))
                            continue;
                        const int slot = atomicAdd(&s_cnt, 1);
                        if (slot >= SPREAD_CAP) {
                            atomicOr(&a.status[4 * d], ST_SPREAD_OVF);
                            continue;
                        }
                        s_node[slot] = j;
                        s_b[0][slot] = r.bx;
                        s_b[1][slot] = r.by;
                        s_b[2][slot] = r.bz;
                        for (int k = 0; k < 4; ++k) {
                            s_w[k][slot] = r.wx[k];
                            s_w[4 + k][slot] = r.wy[k];
                            s_w[8 + k][slot] = r.wz[k];
                        }
                        s_phi[0][slot] = r.phi[0];
                        s_phi[1][slot] = r.phi[1];
                        s_phi[2][slot] = r.phi[2];
                    }
                }
        __syncthreads();
        const int cnt = min(s_cnt, SPREAD_CAP);
        // rank sort by node index: contributions are added in increasing j
        for (int e = tid; e < cnt; e += TILE_CELLS) {
            const int key = s_node[e];
            int rank = 0;
            for (int k = 0; k < cnt; ++k)
                rank += s_node[k] < key;
            s_perm[rank] = (short)e;
        }
        __syncthreads();
        const int X = X0 + (tid & 3), Y = Y0 + ((tid >> 2) & 3), Z = Z0 + (tid >> 4);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int k = 0; k < cnt; ++k) {
            const int e = s_perm[k];
            const int dx = per_off(X, s_b[0][e], D.nx);
            const int dy = per_off(Y, s_b[1][e], D.ny);
            const int dz = D.walls ? Z - s_b[2][e] : per_off(Z, s_b[2][e], D.nzf);
            if (dx < -1 || dx > 2 || dy < -1 || dy > 2 || dz < -1 || dz > 2)
                continue;
            const float w = (s_w[dx + 1][e] * s_w[4 + dy + 1][e]) * s_w[8 + dz + 1][e];
            fx += s_phi[0][e] * w;
            fy += s_phi[1][e] * w;
            fz += s_phi[2][e] * w;
        }
        if (X < D.nx && Y < D.ny && Z < D.nzf) {
            const int64_t g = D.cell0 + X + (int64_t)D.nx * (Y + (int64_t)D.ny * Z);
            a.F[g] = fx;
            a.F[a.total_cells + g] = fy;
            a.F[2 * a.total_cells + g] = fz;
        }
        __syncthreads();
    }
}

// 16 lanes per node: lane l covers support row (dy, dz) = (l & 3, l >> 2)
// and the four cells of that row; partial sums meet in a fixed shuffle tree.
__global__ void interp_advect_kernel(Arrays a)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = gid >> 4, l = gid & 15;
    const bool valid = j < a.total_nodes;
    float ax = 0.f, ay = 0.f, az = 0.f;
    int d = 0;
    if (valid) {
        d = a.node_drop[j];
        const Drop &D = a.drops[d];
        const NodeRec &r = a.rec[j];
        if (r.key >= 0) {
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
                const int64_t row = D.cell0 + (int64_t)D.nx * (Y + (int64_t)D.ny * Z);
                for (int dx = 0; dx < 4; ++dx) {
                    const int64_t g = row + wrapi(r.bx - 1 + dx, D.nx);
                    const float w = r.wx[dx] * wyz;
                    ax += a.U[g] * w;
                    ay += a.U[a.total_cells + g] * w;
                    az += a.U[2 * a.total_cells + g] * w;
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
        a.qx[j] += (double)ax;
        a.qy[j] += (double)ay;
        a.qz[j] += (double)az;
    }
}

}  // namespace

cudaError_t launch_node_force(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    node_force_kernel<<<(a.total_nodes + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_spread(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    scan_blocks_kernel<<<a.n_scan_blocks, 1024, 0, s>>>(a.bin_cnt, a.total_tiles + 1, a.bin_off, a.blk_sum);
    scan_top_kernel<<<1, 1024, 0, s>>>(a.blk_sum, a.n_scan_blocks, a.blk_off);
    fill_kernel<<<(a.total_nodes + 127) / 128, 128, 0, s>>>(a);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    spread_kernel<<<sms * 16, TILE_CELLS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_interp_advect(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    const int64_t threads = (int64_t)a.total_nodes * 16;
    interp_advect_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace iblb
