// fields.cu -- conversion of one droplet's lattice state between the
// context's storage (offsets s_i = f_i - w_i rho0 in FP32 / FP16 / BF16) and
// FP64 arrays in the API layout, plus the derived fields returned to users:
// rho and U from the post-collision state (eq. hydro_var2 of the last step),
// the force density of the last step and the in/out flag of every cell.
#include "iblb_internal.h"

namespace iblb {

namespace {

__constant__ double kW[Q] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                             1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
__constant__ int kC[Q][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                             {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                             {-1, 1, 0}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
                             {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}};

template <typename S> __device__ __forceinline__ double to_d(S v);
template <> __device__ __forceinline__ double to_d<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__half>(__half v) { return (double)__half2float(v); }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <typename S> __device__ __forceinline__ S from_d(double v);
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __half from_d<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

// storage index of population k of compact cell c (rows padded to the pitch)
__device__ __forceinline__ int64_t pop_index(const Drop &D, int k, int64_t c)
{
    const int64_t row = c / D.nx, x = c - row * D.nx;
    return (int64_t)Q * D.pcell0 + (int64_t)k * D.pcells + x + (int64_t)D.pitch * row;
}

template <typename S>
__global__ void export_pop_kernel(Arrays a, int d, const S *f, double *out)
{
    const Drop &D = a.drops[d];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Q * D.cells)
        return;
    const int k = (int)(i / D.cells);
    out[i] = kW[k] * (double)D.rho0 + to_d<S>(f[pop_index(D, k, i - k * D.cells)]);
}

template <typename S>
__global__ void import_pop_kernel(Arrays a, int d, S *f, const double *in)
{
    const Drop &D = a.drops[d];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Q * D.cells)
        return;
    const int k = (int)(i / D.cells);
    f[pop_index(D, k, i - k * D.cells)] = from_d<S>(in[i] - kW[k] * (double)D.rho0);
}

// offsets 0 everywhere (rest state f_i = w_i rho0), padding included
template <typename S>
__global__ void init_pop_kernel(Arrays a, S *f)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Q * a.total_pcells)
        f[i] = from_d<S>(0.0);
}

__device__ __forceinline__ bool band_cell(const Arrays &a, const Drop &D, int64_t c, int *xyz)
{
    const int ci = (int)c;
    const int x = ci % D.nx, y = (ci / D.nx) % D.ny, z = ci / (D.nx * D.ny);
    xyz[0] = x;
    xyz[1] = y;
    xyz[2] = z;
    const int64_t t = D.tile0 + (x >> 2) + (int64_t)D.tx * ((y >> 2) + (int64_t)D.ty * (z >> 2));
    return a.tile_gen[t] == *a.gen;
}

template <typename S>
__global__ void macros_kernel(Arrays a, int d, const S *f, double *rho, double *u)
{
    const Drop &D = a.drops[d];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.cells)
        return;
    double r = D.rho0, j[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < Q; ++k) {
        const double s = to_d<S>(f[pop_index(D, k, c)]);
        r += s;
        for (int e = 0; e < 3; ++e)
            j[e] += kC[k][e] * s;
    }
    int xyz[3];
    double F[3] = {D.bf[0], D.bf[1], D.bf[2]};
    if (band_cell(a, D, c, xyz))
        for (int e = 0; e < 3; ++e)
            F[e] += a.F[e * a.total_pcells + pop_index(D, 0, c) - (int64_t)Q * D.pcell0 + D.pcell0];
    rho[c] = r;
    // post-collision momentum = sum c_i f_i + F (BGK keeps rho U, Guo adds (1-1/2tau) F)
    for (int e = 0; e < 3; ++e)
        u[e * D.cells + c] = (j[e] - 0.5 * F[e]) / r;
}

__global__ void force_kernel(Arrays a, int d, double *F)
{
    const Drop &D = a.drops[d];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.cells)
        return;
    int xyz[3];
    const bool band = band_cell(a, D, c, xyz);
    const int64_t g = pop_index(D, 0, c) - (int64_t)Q * D.pcell0 + D.pcell0;   // padded field index
    for (int e = 0; e < 3; ++e)
        F[e * D.cells + c] = (double)D.bf[e] + (band ? (double)a.F[e * a.total_pcells + g] : 0.0);
}

__global__ void inside_kernel(Arrays a, int d, uint8_t *inside)
{
    const Drop &D = a.drops[d];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.cells)
        return;
    const int ci = (int)c;
    const int x = ci % D.nx, y = (ci / D.nx) % D.ny, z = ci / (D.nx * D.ny);
    int par = 0;
    if (D.vartau) {
        const int64_t col = D.col0 + x + (int64_t)D.nx * y;
        const int cnt = min(a.col_cnt[col], MAXC);
        const double Z = (double)(z + D.walls);
        for (int k = 0; k < cnt; ++k)
            par ^= a.col_z[col * MAXC + k] < Z;
    }
    inside[c] = (uint8_t)par;
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_export_populations(const Arrays &a, int d, int storage, const void *f, double *out,
                                      int64_t cells, cudaStream_t s)
{
    const unsigned g = blocks_for(Q * cells, 256);
    switch (storage) {
    case 0: export_pop_kernel<float><<<g, 256, 0, s>>>(a, d, (const float *)f, out); break;
    case 1: export_pop_kernel<__half><<<g, 256, 0, s>>>(a, d, (const __half *)f, out); break;
    case 2: export_pop_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(a, d, (const __nv_bfloat16 *)f, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_import_populations(const Arrays &a, int d, int storage, void *f, const double *in,
                                      int64_t cells, cudaStream_t s)
{
    const unsigned g = blocks_for(Q * cells, 256);
    switch (storage) {
    case 0: import_pop_kernel<float><<<g, 256, 0, s>>>(a, d, (float *)f, in); break;
    case 1: import_pop_kernel<__half><<<g, 256, 0, s>>>(a, d, (__half *)f, in); break;
    case 2: import_pop_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(a, d, (__nv_bfloat16 *)f, in); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_init_populations(const Arrays &a, int storage, void *f, cudaStream_t s)
{
    const unsigned g = blocks_for(Q * a.total_pcells, 256);
    switch (storage) {
    case 0: init_pop_kernel<float><<<g, 256, 0, s>>>(a, (float *)f); break;
    case 1: init_pop_kernel<__half><<<g, 256, 0, s>>>(a, (__half *)f); break;
    case 2: init_pop_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(a, (__nv_bfloat16 *)f); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_macros(const Arrays &a, int d, int storage, const void *f, double *rho, double *u,
                                 int64_t cells, cudaStream_t s)
{
    const unsigned g = blocks_for(cells, 256);
    switch (storage) {
    case 0: macros_kernel<float><<<g, 256, 0, s>>>(a, d, (const float *)f, rho, u); break;
    case 1: macros_kernel<__half><<<g, 256, 0, s>>>(a, d, (const __half *)f, rho, u); break;
    case 2: macros_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(a, d, (const __nv_bfloat16 *)f, rho, u); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_force(const Arrays &a, int d, double *F, int64_t cells, cudaStream_t s)
{
    force_kernel<<<blocks_for(cells, 256), 256, 0, s>>>(a, d, F);
    return cudaGetLastError();
}

cudaError_t launch_export_inside(const Arrays &a, int d, uint8_t *inside, int64_t cells, cudaStream_t s)
{
    inside_kernel<<<blocks_for(cells, 256), 256, 0, s>>>(a, d, inside);
    return cudaGetLastError();
}

}  // namespace iblb
