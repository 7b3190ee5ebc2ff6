// reduce.cu -- FP64 reductions over the membrane and the lattice:
//   * mesh volume V = (1/6) sum_t q_a . (q_b x q_c), area, node centroid,
//     z_min and z_max (the half-height l = (z_max - z_min)/2 of App. C, eq. ell);
//   * contact-radius protocols (i) and (ii) of Sec. III B;
//   * lattice mass sum_x sum_i f_i: each cell's 19 stored offsets are added
//     in FP32 (a few rounding errors of the offsets' size, about 1e-3 of a
//     cell's density) and the cells in FP64 in a fixed order and tree.
// Every reduction uses a fixed assignment of items to threads and a fixed
// shuffle tree, so results are bitwise reproducible and a droplet's values
// do not depend on the other droplets of a batch.
#include <math.h>

#include <algorithm>

#include "iblb_internal.h"
#include "reduce_util.cuh"

namespace iblb {

struct MeshView {
    const double *qx, *qy, *qz;  // node j at q*[j * stride]
    int stride;
    const int *tri;              // this droplet's faces (node indices into q*)
    int ntri;
    int node0, nnodes;           // this droplet's node range
    int fpc, npc;                // faces and nodes per reduction chunk (mesh_chunks)
    const uint8_t *clamped;      // per node (global index): clamped by the near-wall guard, or nullptr
};

namespace {

constexpr int RB = 256;          // threads per reduction block

// Chunks of a mesh for the observation passes: enough for every SM to
// share the FP64 work (at least RED_MIN_FACES faces and RED_MIN_NODES nodes
// a chunk), at most RED_MAX_CHUNKS (the allocation-free scratch's size);
// the split depends on the mesh's size alone, so results are reproducible.
constexpr int RED_MIN_FACES = 64, RED_MIN_NODES = 32, RED_MAX_CHUNKS = 512;
int mesh_chunks(int nnodes, int ntri, int &fpc, int &npc)
{
    int nc = std::max((ntri + RED_MIN_FACES - 1) / RED_MIN_FACES, (nnodes + RED_MIN_NODES - 1) / RED_MIN_NODES);
    nc = std::min(std::max(nc, 1), RED_MAX_CHUNKS);
    fpc = std::max((ntri + nc - 1) / nc, 1);
    npc = std::max((nnodes + nc - 1) / nc, 1);
    return nc;
}

// chunk k of a mesh: faces [k*fpc, ...) and nodes [k*npc, ...)
// -> 6V, area, sum x, sum y, sum z, z_min, z_max, clamped nodes
__device__ void pass1_chunk(const MeshView &m, int k, double *out)
{
    const int KIND[8] = {0, 0, 0, 0, 0, 1, 2, 0};
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY, 0.0};
    const int f1 = min(m.ntri, (k + 1) * m.fpc);
    for (int t = k * m.fpc + threadIdx.x; t < f1; t += RB) {
        const int ia = m.tri[3 * t] * m.stride, ib = m.tri[3 * t + 1] * m.stride, ic = m.tri[3 * t + 2] * m.stride;
        const double ax = m.qx[ia], ay = m.qy[ia], az = m.qz[ia];
        const double bx = m.qx[ib], by = m.qy[ib], bz = m.qz[ib];
        const double cx = m.qx[ic], cy = m.qy[ic], cz = m.qz[ic];
        v[0] += ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
        const double e1x = bx - ax, e1y = by - ay, e1z = bz - az, e2x = cx - ax, e2y = cy - ay, e2z = cz - az;
        const double Nx = e1y * e2z - e1z * e2y, Ny = e1z * e2x - e1x * e2z, Nz = e1x * e2y - e1y * e2x;
        v[1] += 0.5 * sqrt(Nx * Nx + Ny * Ny + Nz * Nz);
    }
    const int n1 = min(m.nnodes, (k + 1) * m.npc);
    for (int j = k * m.npc + threadIdx.x; j < n1; j += RB) {
        const int ij = (m.node0 + j) * m.stride;
        if (m.clamped)
            v[7] += (double)m.clamped[m.node0 + j];
        v[2] += m.qx[ij];
        v[3] += m.qy[ij];
        const double z = m.qz[ij];
        v[4] += z;
        v[5] = fmin(v[5], z);
        v[6] = fmax(v[6], z);
    }
    block_reduce<8, RB>(v, KIND);
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i)
            out[i] = v[i];
}

// Fold the chunks of droplet blockIdx.x (one warp; chunk i goes to lane i % 32,
// lanes add their chunks in order, then a fixed shuffle tree).  Writes
// V, A, cx, cy, cz, zmin, zmax, clamped nodes.
__device__ void fold_chunks(const double *part, int nch, int nnodes, double *out)
{
    const int lane = threadIdx.x;
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY, 0.0};
    for (int i = lane; i < nch; i += 32) {
        const double *p = part + (int64_t)NRED * i;
        for (int k = 0; k < 5; ++k)
            v[k] += p[k];
        v[5] = fmin(v[5], p[5]);
        v[6] = fmax(v[6], p[6]);
        v[7] += p[7];
    }
    for (int k = 0; k < 5; ++k)
        v[k] = warp_sum(v[k]);
    v[5] = warp_min(v[5]);
    v[6] = warp_max(v[6]);
    v[7] = warp_sum(v[7]);
    if (lane == 0) {
        out[0] = v[0] / 6.0;
        out[1] = v[1];
        out[2] = v[2] / nnodes;
        out[3] = v[3] / nnodes;
        out[4] = v[4] / nnodes;
        out[5] = v[5];
        out[6] = v[6];
        out[7] = v[7];
    }
}

// --- observation of one mesh (view), used by iblb_observe and the stateless
//     entry point.  scratch layout (doubles): [0, NRED*nch) chunk partials,
//     then 8 result slots R: V, A, cx, cy, cz, zmin, zmax, clamped, then protocol
//     partials.

__global__ void __launch_bounds__(RB) pass1_view_kernel(MeshView m, double *part)
{
    griddep_wait();
    pass1_chunk(m, blockIdx.x, part + (int64_t)NRED * blockIdx.x);
}

__global__ void fold_view_kernel(MeshView m, const double *part, int nch, double *R)
{
    griddep_wait();
    fold_chunks(part, nch, m.nnodes, R);
}

// protocol (i): edges (a < b) crossing z = zp: sum of crossing x, y and count;
// protocol (ii): lower-half faces with max |dz| < eps: area.
__global__ void __launch_bounds__(RB) pass2_view_kernel(MeshView m, const double *R, double zp, double flat,
                                                        double *part)
{
    griddep_wait();
    const int KIND[4] = {0, 0, 0, 0};
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const double zmid = 0.5 * (R[5] + R[6]);
    const int k = blockIdx.x;
    const int f1 = min(m.ntri, (k + 1) * m.fpc);
    for (int t = k * m.fpc + threadIdx.x; t < f1; t += RB) {
        int idx[3] = {m.tri[3 * t], m.tri[3 * t + 1], m.tri[3 * t + 2]};
        double zz[3];
        for (int e = 0; e < 3; ++e)
            zz[e] = m.qz[idx[e] * m.stride];
        for (int e = 0; e < 3; ++e) {
            const int ia = idx[e], ib = idx[(e + 1) % 3];
            if (ia > ib)
                continue;
            const double za = zz[e], zb = zz[(e + 1) % 3];
            if (!((za < zp && zb >= zp) || (zb < zp && za >= zp)))
                continue;
            const double s = (zp - za) / (zb - za);
            const double xa = m.qx[ia * m.stride], ya = m.qy[ia * m.stride];
            v[0] += xa + s * (m.qx[ib * m.stride] - xa);
            v[1] += ya + s * (m.qy[ib * m.stride] - ya);
            v[2] += 1.0;
        }
        if ((zz[0] + zz[1] + zz[2]) / 3.0 < zmid) {
            const double dz = fmax(fabs(zz[0] - zz[1]), fmax(fabs(zz[1] - zz[2]), fabs(zz[0] - zz[2])));
            if (dz < flat) {
                const int ia = idx[0] * m.stride, ib = idx[1] * m.stride, ic = idx[2] * m.stride;
                const double e1x = m.qx[ib] - m.qx[ia], e1y = m.qy[ib] - m.qy[ia], e1z = zz[1] - zz[0];
                const double e2x = m.qx[ic] - m.qx[ia], e2y = m.qy[ic] - m.qy[ia], e2z = zz[2] - zz[0];
                const double Nx = e1y * e2z - e1z * e2y, Ny = e1z * e2x - e1x * e2z, Nz = e1x * e2y - e1y * e2x;
                v[3] += 0.5 * sqrt(Nx * Nx + Ny * Ny + Nz * Nz);
            }
        }
    }
    block_reduce<4, RB>(v, KIND);
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i)
            part[4 * k + i] = v[i];
}

// protocol (i) second pass: sum of distances of the crossings from their centre
__global__ void __launch_bounds__(RB) pass3_view_kernel(MeshView m, double zp, const double *C, double *part)
{
    griddep_wait();
    const int KIND[1] = {0};
    double v[1] = {0.0};
    const double cx = C[0], cy = C[1];
    const int k = blockIdx.x;
    const int f1 = min(m.ntri, (k + 1) * m.fpc);
    for (int t = k * m.fpc + threadIdx.x; t < f1; t += RB)
        for (int e = 0; e < 3; ++e) {
            const int ia = m.tri[3 * t + e], ib = m.tri[3 * t + (e + 1) % 3];
            if (ia > ib)
                continue;
            const double za = m.qz[ia * m.stride], zb = m.qz[ib * m.stride];
            if (!((za < zp && zb >= zp) || (zb < zp && za >= zp)))
                continue;
            const double s = (zp - za) / (zb - za);
            const double xa = m.qx[ia * m.stride], ya = m.qy[ia * m.stride];
            const double px = xa + s * (m.qx[ib * m.stride] - xa) - cx;
            const double py = ya + s * (m.qy[ib * m.stride] - ya) - cy;
            v[0] += sqrt(px * px + py * py);
        }
    block_reduce<1, RB>(v, KIND);
    if (threadIdx.x == 0)
        part[k] = v[0];
}

// fold nch groups of `width` partials (one warp, fixed order) into out[width];
// with center != NULL also writes the crossing centre (sum x / count, sum y / count)
__global__ void fold_sums_kernel(const double *part, int nch, int width, double *out, double *center)
{
    griddep_wait();
    const int lane = threadIdx.x;
    for (int k = 0; k < width; ++k) {
        double v = 0.0;
        for (int i = lane; i < nch; i += 32)
            v += part[(int64_t)width * i + k];
        v = warp_sum(v);
        if (lane == 0)
            out[k] = v;
    }
    if (center && lane == 0) {
        center[0] = out[2] > 0.0 ? out[0] / out[2] : 0.0;
        center[1] = out[2] > 0.0 ? out[1] / out[2] : 0.0;
    }
}

// ---- lattice mass: sum over cells of sum_i s_i (FP64), per droplet
template <typename S>
__device__ __forceinline__ float tof(S v);
template <> __device__ __forceinline__ float tof<float>(float v) { return v; }
template <> __device__ __forceinline__ float tof<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ int find_drop_mass(const Drop *D, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].mass_block0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// block b: cells [(b - mass_block0) MASS_CELLS_PER_BLOCK, ...) of its
// droplet, MASS_CELLS_PER_BLOCK / RB per thread (added in FP64 in a fixed
// order), then the fixed block tree: a quarter of the FP64 tree work per
// cell of one cell per thread.
template <typename S>
__global__ void __launch_bounds__(RB) mass_kernel(Arrays a, const S *f)
{
    griddep_wait();
    constexpr int CPT = MASS_CELLS_PER_BLOCK / RB;
    static_assert(CPT * RB == MASS_CELLS_PER_BLOCK, "whole cells per thread");
    const int KIND[1] = {0};
    const int b = blockIdx.x;
    const int d = find_drop_mass(a.drops, a.ndrops, b);
    const Drop &D = a.drops[d];
    const int64_t cb = (int64_t)(b - D.mass_block0) * MASS_CELLS_PER_BLOCK + threadIdx.x;
    float cell[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
        const int64_t c = cb + (int64_t)u * RB;
        cell[u] = 0.0f;
        if (c < D.cells) {
            const int64_t row = c / D.nx;
            const S *p = f + (int64_t)Q * D.pcell0 + (c - row * D.nx) + (int64_t)D.pitch * row;
            for (int i = 0; i < Q; ++i)
                cell[u] += tof<S>(p[(int64_t)i * D.pcells]);
        }
    }
    double v[1] = {0.0};
#pragma unroll
    for (int u = 0; u < CPT; ++u)
        v[0] += (double)cell[u];
    block_reduce<1, RB>(v, KIND);
    if (threadIdx.x == 0)
        a.mass_part[b] = v[0];
}

// one block of RB threads per droplet: thread t adds partials t, t + RB, ...,
// then the fixed block tree
__global__ void __launch_bounds__(RB) mass_fold_kernel(Arrays a, double *out)
{
    griddep_wait();
    const int KIND[1] = {0};
    const Drop &D = a.drops[blockIdx.x];
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < D.mass_nblocks; i += RB)
        v[0] += a.mass_part[D.mass_block0 + i];
    block_reduce<1, RB>(v, KIND);
    if (threadIdx.x == 0)
        out[blockIdx.x] = v[0] + (double)D.rho0 * (double)D.cells;
}

}  // namespace


// scratch: at least NRED*nch + 32 + 4*nch + nch doubles
// Enqueue the observation of a mesh on s: the three passes and their folds,
// then a copy of the 32 result doubles to hv (host; pinned for an
// asynchronous copy).  observe_view_finish turns them into the observables
// once s has reached that point.
static cudaError_t observe_view_enqueue(MeshView m, double R0, double zcut_frac, double eps_flat, double *scr,
                                        double *hv, cudaStream_t s)
{
    const int nc = mesh_chunks(m.nnodes, m.ntri, m.fpc, m.npc);
    double *part1 = scr;                    // NRED * nc
    double *R = scr + (int64_t)NRED * nc;  // 8 results
    double *S2 = R + 8;                     // 4 protocol sums
    double *Cc = S2 + 4;                    // crossing centre (2)
    double *S3 = Cc + 2;                    // 1
    double *part2 = R + 32;                 // 4 * nc
    double *part3 = part2 + 4 * (int64_t)nc;  // nc
    const double zp = 0.5 + zcut_frac * R0;
    const double flat = eps_flat * R0;
    // chained by programmatic dependent launch: each kernel waits for the
    // previous one before reading its results
    cudaError_t e;
    if ((e = launch_k(pass1_view_kernel, dim3(nc), dim3(RB), 0, s, true, m, part1)) != cudaSuccess ||
        (e = launch_k(fold_view_kernel, dim3(1), dim3(32), 0, s, true, m, (const double *)part1, nc, R)) !=
            cudaSuccess ||
        (e = launch_k(pass2_view_kernel, dim3(nc), dim3(RB), 0, s, true, m, (const double *)R, zp, flat, part2)) !=
            cudaSuccess ||
        (e = launch_k(fold_sums_kernel, dim3(1), dim3(32), 0, s, true, (const double *)part2, nc, 4, S2, Cc)) !=
            cudaSuccess ||
        (e = launch_k(pass3_view_kernel, dim3(nc), dim3(RB), 0, s, true, m, zp, (const double *)Cc, part3)) !=
            cudaSuccess ||
        (e = launch_k(fold_sums_kernel, dim3(1), dim3(32), 0, s, true, (const double *)part3, nc, 1, S3,
                      (double *)nullptr)) != cudaSuccess)
        return e;
    return cudaMemcpyAsync(hv, R, sizeof(double) * 32, cudaMemcpyDeviceToHost, s);
}

// h_out: V, A, cx, cy, cz, zmin, zmax, theta(R0), theta(R_V), rc_cut,
// rc_flat, n_cut, chi_flat, clamped nodes
static void observe_view_finish(const double *hv, double R0, double *h_out)
{
    // hv: R[0..7], S2 at 8..11, Cc at 12..13, S3 at 14
    const double V = hv[0], A = hv[1], zmin = hv[5], zmax = hv[6];
    const double ell = 0.5 * (zmax - zmin);
    const double RV = cbrt(3.0 * V / (4.0 * M_PI));
    auto theta = [](double l, double Rr) {
        const double l3 = l * l * l, R3 = Rr * Rr * Rr;
        if (l3 >= R3)
            return 180.0;
        return 2.0 * atan(sqrt(3.0 * l3 / (R3 - l3))) * 180.0 / M_PI;  // eq. angleh
    };
    h_out[0] = V;
    h_out[1] = A;
    h_out[2] = hv[2];
    h_out[3] = hv[3];
    h_out[4] = hv[4];
    h_out[5] = zmin;
    h_out[6] = zmax;
    h_out[7] = theta(ell, R0);
    h_out[8] = theta(ell, RV);
    h_out[9] = hv[10] > 0.0 ? hv[14] / hv[10] : 0.0;  // rc_cut
    h_out[10] = sqrt(hv[11] / M_PI);                  // rc_flat
    h_out[11] = hv[10];                               // n_cut
    h_out[12] = hv[11];                               // chi_flat
    h_out[13] = hv[7];                                // clamped nodes
}

int64_t observe_scratch_doubles(int n_nodes, int n_tri)
{
    int fpc = 0, npc = 0;
    const int nch = mesh_chunks(n_nodes, n_tri, fpc, npc);
    return (int64_t)NRED * nch + 32 + 5 * (int64_t)nch + 8;
}

cudaError_t launch_observe_view(const double *qx, const double *qy, const double *qz, int stride,
                                const int *tri, int ntri, int node0, int nnodes, double R0, double zcut_frac,
                                double eps_flat, double *scratch, double *h_out, cudaStream_t s)
{
    MeshView m{qx, qy, qz, stride, tri, ntri, node0, nnodes, 0, 0, nullptr};
    double hv[32], t[14];
    cudaError_t e = observe_view_enqueue(m, R0, zcut_frac, eps_flat, scratch, hv, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return e;
    observe_view_finish(hv, R0, t);
    for (int i = 0; i < 13; ++i)   // the first 13 (no clamped count for a bare mesh)
        h_out[i] = t[i];
    return cudaSuccess;
}

cudaError_t enqueue_observe(const double *qx, const double *qy, const double *qz, const uint8_t *clamped,
                            const int *tri, int ntri, int node0, int nnodes, double R0, double zcut_frac,
                            double eps_flat, double *scratch, double *hv, cudaStream_t s)
{
    MeshView m{qx, qy, qz, 1, tri, ntri, node0, nnodes, 0, 0, clamped};
    return observe_view_enqueue(m, R0, zcut_frac, eps_flat, scratch, hv, s);
}

void finish_observe(const double *hv, double R0, double *h_out) { observe_view_finish(hv, R0, h_out); }

cudaError_t preload_observe_kernels()
{
    // under lazy module loading a kernel's code reaches the device at its
    // first launch or at the first query of its attributes
    cudaFuncAttributes fa;
    const void *k[] = {(const void *)pass1_view_kernel, (const void *)fold_view_kernel,
                       (const void *)pass2_view_kernel, (const void *)fold_sums_kernel,
                       (const void *)pass3_view_kernel};
    for (const void *f : k) {
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_mass(const Arrays &a, int storage, const void *f, double *d_out, int mass_blocks,
                        cudaStream_t s)
{
    cudaError_t e;
    switch (storage) {
    case 0: e = launch_k(mass_kernel<float>, dim3(mass_blocks), dim3(RB), 0, s, true, a, (const float *)f); break;
    case 1: e = launch_k(mass_kernel<__half>, dim3(mass_blocks), dim3(RB), 0, s, true, a, (const __half *)f); break;
    case 2:
        e = launch_k(mass_kernel<__nv_bfloat16>, dim3(mass_blocks), dim3(RB), 0, s, true, a,
                     (const __nv_bfloat16 *)f);
        break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess)
        return e;
    return launch_k(mass_fold_kernel, dim3(a.ndrops), dim3(RB), 0, s, true, a, d_out);
}

}  // namespace iblb
