// warmstart.cu -- host-side geometry of the learned warm start: the radial
// profile of a droplet mesh about its centre (the App. B parametrisation
// r = G(phi), g = G / R0, phi the polar angle from the z axis, averaged over
// the azimuth as in eq. L2-error_equilibrium), and the inverse map that
// deforms a sphere-like mesh to a given profile before a run starts.
// Neither is part of the time step; both run once per droplet.
#include <math.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/iblb.h"

namespace {

thread_local std::string g_ws_error;

int wfail(int code, const char *msg)
{
    g_ws_error = msg;
    return code;
}

double mesh_volume(const std::vector<double> &q, const int32_t *tri, int n_tri)
{
    double V = 0.0;
    for (int t = 0; t < n_tri; ++t) {
        const double *a = &q[3 * (size_t)tri[3 * t]], *b = &q[3 * (size_t)tri[3 * t + 1]],
                     *c = &q[3 * (size_t)tri[3 * t + 2]];
        V += a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
             a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    return V / 6.0;
}

// linear interpolation of the samples g[k] at phi_k = (k + 1/2) pi / n,
// constant beyond the first and last sample
double profile_at(const double *g, int n, double phi)
{
    const double s = phi / M_PI * n - 0.5;
    if (s <= 0.0)
        return g[0];
    if (s >= n - 1)
        return g[n - 1];
    const int k = (int)s;
    const double f = s - k;
    return (1.0 - f) * g[k] + f * g[k + 1];
}

// Cumulative area of the surface of revolution r(phi) = R0 g(phi) between the
// pole phi = 0 and phi_i = pi i / n (i = 0 .. n), dA = 2 pi r sin(phi)
// sqrt(r^2 + r'^2) dphi, by the midpoint rule on n intervals (r and r' of the
// piecewise-linear profile at the interval midpoints).
void cumulative_area(const double *g, int nphi, double R0, int n, std::vector<double> &A)
{
    A.assign(n + 1, 0.0);
    const double h = M_PI / n;
    for (int i = 0; i < n; ++i) {
        const double phi = (i + 0.5) * h;
        const double r = R0 * profile_at(g, nphi, phi);
        const double dr = R0 * (profile_at(g, nphi, phi + 0.5 * h) - profile_at(g, nphi, phi - 0.5 * h)) / h;
        A[i + 1] = A[i] + 2.0 * M_PI * r * sin(phi) * sqrt(r * r + dr * dr) * h;
    }
}

constexpr int kAreaSteps = 4096;

// polar angle on the target surface below which lies the area fraction f
double angle_at_fraction(const std::vector<double> &A, double f)
{
    const int n = (int)A.size() - 1;
    const double t = f * A[n];
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (A[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    const double w = A[hi] > A[lo] ? (t - A[lo]) / (A[hi] - A[lo]) : 0.0;
    return M_PI * (lo + w) / n;
}

}  // namespace

extern "C" {

const char *iblb_warmstart_last_error(void) { return g_ws_error.c_str(); }

int iblb_mesh_profile(const double *xyz, int n_nodes, double R0, int nphi, double *g)
{
    if (!xyz || !g || n_nodes < 1 || !(R0 > 0.0) || nphi < 2)
        return wfail(IBLB_E_ARG, "iblb_mesh_profile: bad arguments");
    double c[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < n_nodes; ++j)
        for (int a = 0; a < 3; ++a)
            c[a] += xyz[3 * (size_t)j + a];
    for (int a = 0; a < 3; ++a)
        c[a] /= n_nodes;
    std::vector<double> sum(nphi, 0.0);
    std::vector<int> cnt(nphi, 0);
    for (int j = 0; j < n_nodes; ++j) {
        const double dx = xyz[3 * (size_t)j] - c[0], dy = xyz[3 * (size_t)j + 1] - c[1],
                     dz = xyz[3 * (size_t)j + 2] - c[2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r > 0.0) || !std::isfinite(r))
            continue;
        const double phi = acos(fmax(-1.0, fmin(1.0, dz / r)));
        int k = (int)(phi / M_PI * nphi);
        k = k < 0 ? 0 : (k >= nphi ? nphi - 1 : k);
        sum[k] += r;
        cnt[k] += 1;
    }
    int first = -1;
    for (int k = 0; k < nphi; ++k)
        if (cnt[k]) {
            g[k] = sum[k] / cnt[k] / R0;
            if (first < 0)
                first = k;
        }
    if (first < 0)
        return wfail(IBLB_E_MESH, "iblb_mesh_profile: every node sits at the centroid");
    // empty bins: linear interpolation between the nearest filled bins
    // (constant beyond the first and the last filled bin)
    int prev = -1;
    for (int k = 0; k < nphi; ++k) {
        if (cnt[k]) {
            prev = k;
            continue;
        }
        int next = k + 1;
        while (next < nphi && !cnt[next])
            ++next;
        if (prev < 0)
            g[k] = g[next];
        else if (next >= nphi)
            g[k] = g[prev];
        else
            g[k] = g[prev] + (g[next] - g[prev]) * (double)(k - prev) / (double)(next - prev);
    }
    return IBLB_OK;
}

int iblb_deform_mesh(const double *g, int nphi, double R0, const double *xyz, int n_nodes, const int32_t *tri,
                     int n_tri, double cx, double cy, double z_bottom, double *xyz_out)
{
    if (!g || !xyz || !tri || !xyz_out || nphi < 2 || n_nodes < 4 || n_tri < 4 || !(R0 > 0.0))
        return wfail(IBLB_E_ARG, "iblb_deform_mesh: bad arguments");
    for (int k = 0; k < nphi; ++k)
        if (!(g[k] > 0.0) || !std::isfinite(g[k]))
            return wfail(IBLB_E_ARG, "iblb_deform_mesh: the profile must be positive and finite");
    for (int t = 0; t < 3 * n_tri; ++t)
        if (tri[t] < 0 || tri[t] >= n_nodes)
            return wfail(IBLB_E_MESH, "iblb_deform_mesh: face index out of range");
    double c[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < n_nodes; ++j)
        for (int a = 0; a < 3; ++a)
            c[a] += xyz[3 * (size_t)j + a];
    for (int a = 0; a < 3; ++a)
        c[a] /= n_nodes;
    std::vector<double> area;
    cumulative_area(g, nphi, R0, kAreaSteps, area);
    std::vector<double> q0(3 * (size_t)n_nodes), q(3 * (size_t)n_nodes);
    for (int j = 0; j < n_nodes; ++j) {
        double d[3], r = 0.0;
        for (int a = 0; a < 3; ++a) {
            d[a] = xyz[3 * (size_t)j + a] - c[a];
            r += d[a] * d[a];
        }
        r = sqrt(r);
        if (!(r > 0.0))
            return wfail(IBLB_E_MESH, "iblb_deform_mesh: a node sits at the centroid");
        for (int a = 0; a < 3; ++a)
            q0[3 * (size_t)j + a] = d[a];
        // the node keeps its azimuth and its area fraction from the pole:
        // on the unit sphere the fraction below polar angle phi is
        // (1 - cos phi) / 2
        const double cs = fmax(-1.0, fmin(1.0, d[2] / r));
        const double phi = angle_at_fraction(area, 0.5 * (1.0 - cs));
        const double rho = sqrt(d[0] * d[0] + d[1] * d[1]);
        const double ca = rho > 0.0 ? d[0] / rho : 1.0, sa = rho > 0.0 ? d[1] / rho : 0.0;
        const double G = R0 * profile_at(g, nphi, phi);
        q[3 * (size_t)j] = G * sin(phi) * ca;
        q[3 * (size_t)j + 1] = G * sin(phi) * sa;
        q[3 * (size_t)j + 2] = G * cos(phi);
    }
    const double V0 = mesh_volume(q0, tri, n_tri), V = mesh_volume(q, tri, n_tri);
    if (!(V0 > 0.0) || !(V > 0.0))
        return wfail(IBLB_E_MESH, "iblb_deform_mesh: the mesh must enclose a positive volume before and after");
    const double s = cbrt(V0 / V);
    double zmin = INFINITY;
    for (int j = 0; j < n_nodes; ++j)
        zmin = fmin(zmin, s * q[3 * (size_t)j + 2]);
    for (int j = 0; j < n_nodes; ++j) {
        xyz_out[3 * (size_t)j] = cx + s * q[3 * (size_t)j];
        xyz_out[3 * (size_t)j + 1] = cy + s * q[3 * (size_t)j + 1];
        xyz_out[3 * (size_t)j + 2] = z_bottom + (s * q[3 * (size_t)j + 2] - zmin);
    }
    return IBLB_OK;
}

int iblb_cap_profile(double theta_eq_deg, int nphi, double *g)
{
    if (!g || nphi < 2 || !(theta_eq_deg > 0.0) || !(theta_eq_deg < 180.0))
        return wfail(IBLB_E_ARG, "iblb_cap_profile: bad arguments");
    const double th = theta_eq_deg * M_PI / 180.0, c = cos(th);
    const double rho = cbrt(4.0 / (2.0 - 3.0 * c + c * c * c));   // radius of the cap's sphere (unit volume sphere)
    const double h = rho * (1.0 - c);                              // cap height above its base z = 0
    const double base = rho * sin(th);
    // surface centroid: the curved part (area 2 pi rho h, its height spread
    // evenly in z, so its mean is h / 2) and the base disc at z = 0
    const double z0 = (2.0 * M_PI * rho * h * 0.5 * h) / (2.0 * M_PI * rho * h + M_PI * base * base);
    const double dz = z0 + rho * c;                                // the centroid above the sphere's centre
    for (int k = 0; k < nphi; ++k) {
        const double phi = (k + 0.5) * M_PI / nphi;
        const double ur = sin(phi), uz = cos(phi);
        (void)ur;
        // from the centroid along (sin phi, cos phi): the sphere's far
        // intersection if it lies on the cap, else the base plane z = 0
        const double t_sph = -uz * dz + sqrt(uz * dz * uz * dz - (dz * dz - rho * rho));
        if (z0 + uz * t_sph >= 0.0)
            g[k] = t_sph;
        else
            g[k] = -z0 / uz;
    }
    return IBLB_OK;
}

}  // extern "C"
