// ib.cu -- the membrane side of the IB-LB step:
//   * nodal forces: surface tension phi_sigma,j = -sigma dA/dq_j (Sec. II B)
//     plus the wall interaction phi_Pi,j = -(chi_j/3) Pi(h_j) n_j (Sec. II C);
//     8 lanes per node share its incident faces, partial sums meet in a fixed
//     shuffle tree;
//   * force spreading F(x) = sum_j phi_j Delta(q_j - x) (eq. force_spread) as
//     a deterministic binned gather: every node is listed in the 4^3 tiles its
//     4x4x4 kernel support touches (at most 8, or 27 across a partial periodic
//     tile); the non-empty tiles form the band; every band tile gathers its
//     nodes, orders them by node index and each cell adds their contributions
//     in that order, so the result depends neither on launch shapes nor on the
//     other droplets of a batch;
//   * interpolation qdot_j = sum_x U(x) Delta(q_j - x) (eq. vel_interpolation)
//     and forward-Euler advection q_j += qdot_j, 16 lanes per node.
// Node positions are FP64 so that edge vectors and kernel offsets are exact
// before they are rounded to FP32 for the force and kernel arithmetic.
#include "iblb_internal.h"

namespace iblb {

namespace {

constexpr int FL = 8;          // lanes per node in the force and fill kernels

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

// Distinct tiles (in increasing cell order) holding the support cells
// b-1 .. b+2 of one axis of n cells: wrapped on a periodic axis, clipped to
// [0, n) otherwise.  At most 3 (a partial last tile of a periodic axis).
__device__ __forceinline__ int support_tiles(int b, int n, bool periodic, int *out)
{
    int cnt = 0;
    for (int k = -1; k <= 2; ++k) {
        int c = b + k;
        if (periodic)
            c = wrapi(c, n);
        else if (c < 0 || c >= n)
            continue;
        const int t = c >> 2;
        if (cnt == 0 || out[cnt - 1] != t) {
            bool dup = false;
            for (int i = 0; i < cnt; ++i)
                dup |= out[i] == t;
            if (!dup)
                out[cnt++] = t;
        }
    }
    return cnt;
}

// FL lanes per node; lane l takes the node's incident faces l, l + FL, ...
// Lane 0 writes the node record; the lanes then list the node in the tiles
// its kernel support touches: its slot in a tile's list (TILE_CAP slots per
// tile) comes from the tile's counter, and the node that takes slot 0 stamps
// the tile with this step's generation and appends it to the band list.
// (Nothing in this kernel reads the generation counter's new value; the
// spread kernel commits it.)
__global__ void __launch_bounds__(128) node_force_kernel(Arrays a)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = gid / FL, l = gid % FL;
    const bool valid = j < a.total_nodes;
    float gx = 0.f, gy = 0.f, gz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f, chi = 0.f;
    if (valid) {
        const int e1 = a.adj_start[j + 1];
        for (int e = a.adj_start[j] + l; e < e1; e += FL) {
            const int code = a.adj[e];
            const int t = code >> 2, k = code & 3;
            const int v0 = a.tri[3 * t], v1 = a.tri[3 * t + 1], v2 = a.tri[3 * t + 2];
            const double x0 = a.qx[v0], y0 = a.qy[v0], z0 = a.qz[v0];
            const double x1 = a.qx[v1], y1 = a.qy[v1], z1 = a.qz[v1];
            const double x2 = a.qx[v2], y2 = a.qy[v2], z2 = a.qz[v2];
            const float e1x = (float)(x1 - x0), e1y = (float)(y1 - y0), e1z = (float)(z1 - z0);
            const float e2x = (float)(x2 - x0), e2y = (float)(y2 - y0), e2z = (float)(z2 - z0);
            const float Nx = e1y * e2z - e1z * e2y;
            const float Ny = e1z * e2x - e1x * e2z;
            const float Nz = e1x * e2y - e1y * e2x;
            const float len = sqrtf(Nx * Nx + Ny * Ny + Nz * Nz);
            const float il = 1.0f / len;
            const float hx = Nx * il, hy = Ny * il, hz = Nz * il;
            // dA/dq_k = 1/2 n x (q_prev - q_next), corners in CCW order
            float dx, dy, dz;
            if (k == 0) {
                dx = (float)(x2 - x1); dy = (float)(y2 - y1); dz = (float)(z2 - z1);
            } else if (k == 1) {
                dx = (float)(x0 - x2); dy = (float)(y0 - y2); dz = (float)(z0 - z2);
            } else {
                dx = (float)(x1 - x0); dy = (float)(y1 - y0); dz = (float)(z1 - z0);
            }
            gx += 0.5f * (hy * dz - hz * dy);
            gy += 0.5f * (hz * dx - hx * dz);
            gz += 0.5f * (hx * dy - hy * dx);
            nx += hx;
            ny += hy;
            nz += hz;
            chi += 0.5f * len;
        }
    }
    for (int o = FL / 2; o >= 1; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
        nx += __shfl_xor_sync(0xffffffffu, nx, o);
        ny += __shfl_xor_sync(0xffffffffu, ny, o);
        nz += __shfl_xor_sync(0xffffffffu, nz, o);
        chi += __shfl_xor_sync(0xffffffffu, chi, o);
    }
    if (!valid)
        return;
    const int d = a.node_drop[j];
    const Drop &D = a.drops[d];
    const double qx = a.qx[j], qy = a.qy[j], qz = a.qz[j];
    const bool sane = fabs(qx) < 1e8 && fabs(qy) < 1e8 && fabs(qz) < 1e8;
    int bx = 0, by = 0, bz = 0;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (sane) {
        // support of the 4-point kernel: base-1 .. base+2 on each axis
        const double fbx = floor(qx), fby = floor(qy), fbz = floor(qz);
        fx = (float)(qx - fbx);
        fy = (float)(qy - fby);
        fz = (float)(qz - fbz);
        bx = wrapi((int)fbx % D.nx, D.nx);
        by = wrapi((int)fby % D.ny, D.ny);
        bz = (int)fbz - D.walls;
        if (!D.walls)
            bz = wrapi(bz % D.nz, D.nz);
    }
    // tiles touched by the support (fluid cells only)
    int txs[3], tys[3], tzs[3];
    int ntx = 0, nty = 0, ntz = 0;
    if (sane) {
        ntx = support_tiles(bx, D.nx, true, txs);
        nty = support_tiles(by, D.ny, true, tys);
        ntz = support_tiles(bz, D.nzf, !D.walls, tzs);
    }
    const int ncombo = ntx * nty * ntz;
    if (l == 0) {
        NodeRec r;
        r.bx = bx;
        r.by = by;
        r.bz = bz;
        r.key = ncombo;
        r.spare = d;
        uint8_t clamped = 0;
        if (!sane) {
            atomicOr(&a.status[4 * d], ST_NAN);
            for (int k = 0; k < 4; ++k)
                r.wx[k] = r.wy[k] = r.wz[k] = 0.0f;
            r.phi[0] = r.phi[1] = r.phi[2] = 0.0f;
        } else {
            float px = -D.sigma * gx, py = -D.sigma * gy, pz = -D.sigma * gz;
            if (D.wetting) {
                float h = (float)(qz - 0.5);
                if (h < D.hmin) {
                    h = D.hmin;
                    clamped = 1;
                }
                const float r0 = D.xi / h;
                const float Pi = D.A * (ipow(r0, D.n) - ipow(r0, D.m));
                const float inl = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
                const float s = -(chi * (1.0f / 3.0f)) * Pi * inl;
                px += s * nx;
                py += s * ny;
                pz += s * nz;
            }
            r.wx[0] = psi_far(1.0f + fx); r.wx[1] = psi_near(fx); r.wx[2] = psi_near(1.0f - fx); r.wx[3] = psi_far(2.0f - fx);
            r.wy[0] = psi_far(1.0f + fy); r.wy[1] = psi_near(fy); r.wy[2] = psi_near(1.0f - fy); r.wy[3] = psi_far(2.0f - fy);
            r.wz[0] = psi_far(1.0f + fz); r.wz[1] = psi_near(fz); r.wz[2] = psi_near(1.0f - fz); r.wz[3] = psi_far(2.0f - fz);
            r.phi[0] = px;
            r.phi[1] = py;
            r.phi[2] = pz;
            if (ncombo == 0)
                atomicOr(&a.status[4 * d], ST_ESCAPE);
        }
        a.rec[j] = r;
        a.clamped[j] = clamped;
    }
    // this step's generation (committed by the spread kernel when it ends)
    const uint32_t gen = *a.gen + 1u;
    const int cur = (int)(gen & 1u);
    for (int c = l; c < ncombo; c += FL) {
        const int ix = c % ntx, iy = (c / ntx) % nty, iz = c / (ntx * nty);
        const int64_t t = D.tile0 + txs[ix] + (int64_t)D.tx * (tys[iy] + (int64_t)D.ty * tzs[iz]);
        const int rank = atomicAdd(&a.bin_cnt[t], 1);
        if (rank == 0) {        // first node of the tile: the tile joins the band
            a.tile_gen[t] = gen;
            const int slot = atomicAdd(&a.n_active[cur], 1);
            if (slot < a.active_cap)
                a.active[(int64_t)cur * a.active_cap + slot] = (int)t;
        }
        if (rank < TILE_CAP)
            a.tile_list[t * TILE_CAP + rank] = j;
        else
            atomicOr(&a.status[4 * d], ST_SPREAD_OVF);
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

// One 128-thread block per band tile (block-stride over the band list).  The
// tile's nodes are staged in parallel and sorted by node index; two threads
// per cell add the two halves of the sorted list and the halves are summed
// in a fixed order, so every cell's force is the same for any launch shape.
constexpr int SPREAD_THREADS = 2 * TILE_CELLS;

__global__ void __launch_bounds__(SPREAD_THREADS) spread_kernel(Arrays a)
{
    __shared__ int s_node[SPREAD_CAP];
    __shared__ short s_perm[SPREAD_CAP];
    __shared__ int s_b[3][SPREAD_CAP];
    __shared__ float s_w[12][SPREAD_CAP];
    __shared__ float s_phi[3][SPREAD_CAP];
    __shared__ float s_part[3][TILE_CELLS];
    const uint32_t gen = *a.gen + 1u;          // this step's generation, committed below
    const int cur = (int)(gen & 1u);
    const int nact = min(a.n_active[cur], a.active_cap);
    const int *list = a.active + (int64_t)cur * a.active_cap;
    const int tid = threadIdx.x;
    // tiles that left the band since the previous step: zero their force, so
    // F vanishes outside this step's band (band tiles are rewritten below)
    {
        const int nprev = min(a.n_active[cur ^ 1], a.active_cap);
        const int *plist = a.active + (int64_t)(cur ^ 1) * a.active_cap;
        for (int it = blockIdx.x * 2 + (tid >> 6); it < nprev; it += gridDim.x * 2) {
            const int64_t T = plist[it];
            if (a.tile_gen[T] == gen)
                continue;
            const int d = find_drop_tile(a.drops, a.ndrops, T);
            const Drop &D = a.drops[d];
            const int local = (int)(T - D.tile0), cell = tid & 63;
            const int X = 4 * (local % D.tx) + (cell & 3);
            const int Y = 4 * ((local / D.tx) % D.ty) + ((cell >> 2) & 3);
            const int Z = 4 * (local / (D.tx * D.ty)) + (cell >> 4);
            if (X < D.nx && Y < D.ny && Z < D.nzf) {
                const int64_t g = D.pcell0 + X + (int64_t)D.pitch * (Y + (int64_t)D.ny * Z);
                a.F[g] = 0.0f;
                a.F[a.total_pcells + g] = 0.0f;
                a.F[2 * a.total_pcells + g] = 0.0f;
            }
        }
    }
    for (int it = blockIdx.x; it < nact; it += gridDim.x) {
        const int64_t T = list[it];
        const int d = find_drop_tile(a.drops, a.ndrops, T);
        const Drop &D = a.drops[d];
        const int local = (int)(T - D.tile0);
        const int X0 = 4 * (local % D.tx), Y0 = 4 * ((local / D.tx) % D.ty), Z0 = 4 * (local / (D.tx * D.ty));
        const int64_t e0 = T * TILE_CAP;
        const int cnt = min(a.bin_cnt[T], TILE_CAP);     // overflow was flagged by the force kernel
        for (int e = tid; e < cnt; e += SPREAD_THREADS) {
            const int j = a.tile_list[e0 + e];
            const NodeRec &r = a.rec[j];
            s_node[e] = j;
            s_b[0][e] = r.bx;
            s_b[1][e] = r.by;
            s_b[2][e] = r.bz;
            for (int q = 0; q < 4; ++q) {
                s_w[q][e] = r.wx[q];
                s_w[4 + q][e] = r.wy[q];
                s_w[8 + q][e] = r.wz[q];
            }
            s_phi[0][e] = r.phi[0];
            s_phi[1][e] = r.phi[1];
            s_phi[2][e] = r.phi[2];
        }
        __syncthreads();
        if (tid == 0)
            a.bin_cnt[T] = 0;                            // empty for the next step
        // rank sort by node index: contributions are added in increasing j
        for (int e = tid; e < cnt; e += SPREAD_THREADS) {
            const int key = s_node[e];
            int rank = 0;
            for (int k = 0; k < cnt; ++k)
                rank += s_node[k] < key;
            s_perm[rank] = (short)e;
        }
        __syncthreads();
        const int cell = tid & (TILE_CELLS - 1), part = tid >> 6;
        const int X = X0 + (cell & 3), Y = Y0 + ((cell >> 2) & 3), Z = Z0 + (cell >> 4);
        const int k0 = part ? (cnt >> 1) : 0, k1 = part ? cnt : (cnt >> 1);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int k = k0; k < k1; ++k) {
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
        if (part) {
            s_part[0][cell] = fx;
            s_part[1][cell] = fy;
            s_part[2][cell] = fz;
        }
        __syncthreads();
        if (!part && X < D.nx && Y < D.ny && Z < D.nzf) {
            fx += s_part[0][cell];
            fy += s_part[1][cell];
            fz += s_part[2][cell];
            const int64_t g = D.pcell0 + X + (int64_t)D.pitch * (Y + (int64_t)D.ny * Z);
            a.F[g] = fx;
            a.F[a.total_pcells + g] = fy;
            a.F[2 * a.total_pcells + g] = fz;
        }
        __syncthreads();
    }
    // the last block to finish commits the generation and empties the
    // previous step's band list, which the next step fills
    __shared__ int s_last;
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(a.spread_done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && tid == 0) {
        *a.gen = gen;
        a.n_active[cur ^ 1] = 0;
        *a.spread_done = 0;
    }
}

// 16 lanes per node: lane l covers support row (dy, dz) = (l & 3, l >> 2)
// and the four cells of that row; partial sums meet in a fixed shuffle tree.
__global__ void __launch_bounds__(256) interp_advect_kernel(Arrays a)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = gid >> 4, l = gid & 15;
    const bool valid = j < a.total_nodes;
    float ax = 0.f, ay = 0.f, az = 0.f;
    int d = 0;
    if (valid) {
        const NodeRec &r = a.rec[j];
        d = r.spare;
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
                    ax += a.U[g] * w;
                    ay += a.U[a.total_pcells + g] * w;
                    az += a.U[2 * a.total_pcells + g] * w;
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

int g_sm_count = 0;

}  // namespace

cudaError_t launch_node_force(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    const int64_t threads = (int64_t)a.total_nodes * FL;
    node_force_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_spread(const Arrays &a, cudaStream_t s)
{
    if (a.total_nodes <= 0)
        return cudaSuccess;
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    spread_kernel<<<g_sm_count * 5, SPREAD_THREADS, 0, s>>>(a);
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
