// inout.cu -- in/out classification of lattice cells for the viscosity
// ratio (Sec. II A: tau = tau_in inside the closed interface, tau_out
// outside, re-identified every step by ray tracing).
//
// A vertical ray runs through every lattice column (X, Y).  One thread per
// face finds the columns inside the face's xy projection and records the z of
// the crossing; one thread per column sorts its crossings; a cell is inside
// iff an odd number of crossings lies strictly below it.  Points on a shared
// edge or vertex are assigned by a half-open rule (a symbolic shift of the
// point by (-e, -e^2)) and each edge function is evaluated from its
// lower-numbered end point, so the two faces of an edge see exactly opposite
// values and the surface is watertight.  All decisions are taken in FP64 with
// every product and sum individually rounded (no contraction), i.e. in plain
// IEEE arithmetic.
#include "iblb_internal.h"

namespace iblb {

namespace {

__device__ __forceinline__ double orient_edge(const Arrays &a, int iu, int iv, double px, double py)
{
    const int lo = iu < iv ? iu : iv, hi = iu < iv ? iv : iu;
    const double ax = a.px[lo], ay = a.py[lo], bx = a.px[hi], by = a.py[hi];
    const double e = __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay)),
                               __dmul_rn(__dsub_rn(by, ay), __dsub_rn(px, ax)));
    return iu < iv ? e : -e;
}

__device__ __forceinline__ bool edge_keeps(const Arrays &a, int iu, int iv, bool up)
{
    const int lo = iu < iv ? iu : iv, hi = iu < iv ? iv : iu;
    double dx = __dsub_rn(a.px[hi], a.px[lo]), dy = __dsub_rn(a.py[hi], a.py[lo]);
    if ((iu < iv) != up) {
        dx = -dx;
        dy = -dy;
    }
    return dy > 0.0 || (dy == 0.0 && dx < 0.0);
}

__device__ __forceinline__ double face_orient(const Arrays &a, int v0, int v1, int v2)
{
    int x = v0, y = v1, z = v2, t;
    bool even = true;
    if (x > y) { t = x; x = y; y = t; even = !even; }
    if (y > z) { t = y; y = z; z = t; even = !even; }
    if (x > y) { t = x; x = y; y = t; even = !even; }
    const double D = __dsub_rn(__dmul_rn(__dsub_rn(a.px[y], a.px[x]), __dsub_rn(a.py[z], a.py[x])),
                               __dmul_rn(__dsub_rn(a.py[y], a.py[x]), __dsub_rn(a.px[z], a.px[x])));
    return even ? D : -D;
}

__global__ void clear_cols_kernel(Arrays a)
{
    griddep_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.total_cols)
        a.col_cnt[i] = 0;
}

__global__ void face_cross_kernel(Arrays a)
{
    griddep_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.total_tri)
        return;
    const int d = a.face_drop[t];
    const Drop &D = a.drops[d];
    if (!D.vartau)
        return;
    const int v0 = a.tri[3 * t], v1 = a.tri[3 * t + 1], v2 = a.tri[3 * t + 2];
    for (int k = 0; k < 3; ++k) {
        const int v = k == 0 ? v0 : (k == 1 ? v1 : v2);
        if (!(fabs(a.px[v]) < 1e8 && fabs(a.py[v]) < 1e8 && fabs(a.pz[v]) < 1e8))
            return;   // flagged by the force kernel
    }
    const double Dor = face_orient(a, v0, v1, v2);
    if (Dor == 0.0)
        return;
    const bool up = Dor > 0.0;
    const double xmin = fmin(a.px[v0], fmin(a.px[v1], a.px[v2]));
    const double xmax = fmax(a.px[v0], fmax(a.px[v1], a.px[v2]));
    const double ymin = fmin(a.py[v0], fmin(a.py[v1], a.py[v2]));
    const double ymax = fmax(a.py[v0], fmax(a.py[v1], a.py[v2]));
    const int PX0 = (int)ceil(xmin), PX1 = (int)floor(xmax);
    const int PY0 = (int)ceil(ymin), PY1 = (int)floor(ymax);
    if (PX1 - PX0 > D.nx || PY1 - PY0 > D.ny) {
        // a face wider than the box: the membrane has blown up
        atomicOr(&a.status[4 * d], ST_COL_OVF);
        return;
    }
    for (int PY = PY0; PY <= PY1; ++PY)
        for (int PX = PX0; PX <= PX1; ++PX) {
            const double px = (double)PX, py = (double)PY;
            const double e0 = orient_edge(a, v1, v2, px, py);
            const double e1 = orient_edge(a, v2, v0, px, py);
            const double e2 = orient_edge(a, v0, v1, px, py);
            const bool in0 = (up ? e0 > 0.0 : e0 < 0.0) || (e0 == 0.0 && edge_keeps(a, v1, v2, up));
            const bool in1 = (up ? e1 > 0.0 : e1 < 0.0) || (e1 == 0.0 && edge_keeps(a, v2, v0, up));
            const bool in2 = (up ? e2 > 0.0 : e2 < 0.0) || (e2 == 0.0 && edge_keeps(a, v0, v1, up));
            if (!(in0 && in1 && in2))
                continue;
            const double num = __dadd_rn(__dadd_rn(__dmul_rn(e0, a.pz[v0]), __dmul_rn(e1, a.pz[v1])),
                                         __dmul_rn(e2, a.pz[v2]));
            const double den = __dadd_rn(__dadd_rn(e0, e1), e2);
            const double zc = __ddiv_rn(num, den);
            const int64_t col = D.col0 + wrapi(((PX % D.nx) + D.nx) % D.nx, D.nx) +
                                (int64_t)D.nx * (((PY % D.ny) + D.ny) % D.ny);
            const int slot = atomicAdd(&a.col_cnt[col], 1);
            if (slot < MAXC)
                a.col_z[col * MAXC + slot] = zc;
            else
                atomicOr(&a.status[4 * d], ST_COL_OVF);
        }
}

// insertion sort of the crossings of one column (at most MAXC values)
__global__ void col_sort_kernel(Arrays a)
{
    griddep_wait();
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= a.total_cols)
        return;
    const int n = min(a.col_cnt[col], MAXC);
    if (n < 2)
        return;
    double v[MAXC];
    for (int k = 0; k < MAXC; ++k)
        v[k] = k < n ? a.col_z[col * MAXC + k] : 0.0;
    for (int i = 1; i < n; ++i) {
        const double x = v[i];
        int k = i - 1;
        while (k >= 0 && v[k] > x) {
            v[k + 1] = v[k];
            --k;
        }
        v[k + 1] = x;
    }
    for (int k = 0; k < n; ++k)
        a.col_z[col * MAXC + k] = v[k];
}

}  // namespace

cudaError_t launch_inout(const Arrays &a, cudaStream_t s)
{
    if (a.total_tri <= 0 || a.total_cols <= 0)
        return cudaSuccess;
    const unsigned cb = (unsigned)((a.total_cols + 255) / 256);
    cudaError_t e = launch_k(clear_cols_kernel, dim3(cb), dim3(256), 0, s, a.pdl != 0, a);
    if (e == cudaSuccess)
        e = launch_k(face_cross_kernel, dim3((a.total_tri + 127) / 128), dim3(128), 0, s, a.pdl != 0, a);
    if (e == cudaSuccess)
        e = launch_k(col_sort_kernel, dim3(cb), dim3(256), 0, s, a.pdl != 0, a);
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}

}  // namespace iblb
