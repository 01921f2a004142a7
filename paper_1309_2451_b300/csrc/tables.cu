// tables.cu -- pass geometry and FP64-generated factor tables (host code).
//
// Every twiddle and phase factor is generated in FP64 on the host and
// stored in lifting form {p = -tan(phi/2), u = sin(phi), s = +-1} with
// exp(i a) = s * rotate(phi), |phi| <= pi/2, then rounded once to the plan's
// precision.  Imaginary-time tables carry the real factor in f.
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "plan.hpp"

namespace ctap {

double grid_point(int i, int n, double lo, double hi) { return lo + (double)i * (hi - lo) / n; }

static double wavenumber(int m, int n, double lo, double hi)
{
    int mm = (m < (n + 1) / 2) ? m : m - n;
    if (n == 1) mm = 0;
    return 2.0 * kPi * (double)mm / (hi - lo);
}

static int lg2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// exp(i a) for a = pi * num/den (exact reduction to |phi| <= pi/2)
static void lift_rational(long long num, long long den, double &p, double &u, double &s)
{
    // a/pi = num/den; m = nearest integer; phi = pi (num - m den)/den
    long long m = (long long)std::llround((double)num / (double)den);
    const double phi = kPi * (double)(num - m * den) / (double)den;
    s = (m & 1) ? -1.0 : 1.0;
    p = -std::tan(0.5 * phi);
    u = std::sin(phi);
}

// exp(i a) for a general FP64 angle
static void lift_angle(double a, double &p, double &u, double &s)
{
    const double m = std::nearbyint(a / kPi);
    const double phi = a - m * kPi;
    s = (std::fmod(std::fabs(m), 2.0) == 1.0) ? -1.0 : 1.0;
    p = -std::tan(0.5 * phi);
    u = std::sin(phi);
}

template <class T>
static void put(std::vector<unsigned char> &h, size_t idx, double p, double u, double s, double f)
{
    Lift<T> L{(T)p, (T)u, (T)s, (T)f};
    std::memcpy(h.data() + idx * sizeof(Lift<T>), &L, sizeof(L));
}

static void put_any(const PlanState &st, std::vector<unsigned char> &h, size_t idx, double p,
                    double u, double s, double f)
{
    if (st.dtype == CTAP_C64) put<float>(h, idx, p, u, s, f);
    else if (st.dtype == CTAP_C128_DF) put<df>(h, idx, p, u, s, f);
    else put<double>(h, idx, p, u, s, f);
}

static size_t lift_size(const PlanState &st)
{
    if (st.dtype == CTAP_C64) return sizeof(Lift<float>);
    return st.dtype == CTAP_C128_DF ? sizeof(Lift<df>) : sizeof(Lift<double>);
}

static AxisPlan make_axis(int L, int maxv, int &table_entries)
{
    AxisPlan ap{};
    ap.lgL = lg2(L);
    int rem = L, lgNs = 0;
    ap.nst = 0;
    while (rem > 1) {
        int R = rem < maxv ? rem : maxv;
        ap.R[ap.nst] = R;
        ap.lgNs[ap.nst] = lgNs;
        if (lgNs > 0) {
            ap.off[ap.nst] = table_entries;
            table_entries += (1 << lgNs) * R;
        } else {
            ap.off[ap.nst] = 0;
        }
        lgNs += lg2(R);
        rem /= R;
        ++ap.nst;
    }
    return ap;
}

void build_geometry(PlanState &p, int emax, int maxv)
{
    Geom &g = p.geom;
    std::memset(&g, 0, sizeof(g));
    g.nx = p.nx;
    g.ny = p.ny;
    g.nz = p.nz;
    int P = 1;
    while ((long long)p.nx * p.ny / P > emax) P *= 2;
    p.fast_xy = false;
    p.fast_z = false;
    const int LYF = fast_rows(p.esize);
    if (!p.force_generic && p.ny >= LYF && fast_xy_supported(p.esize, p.nx, LYF) &&
        p.ny / LYF <= 16) {
        P = p.ny / LYF;                      // row classes of the specialised XY pass
        p.fast_xy = true;
    }
    if (P > 16 || P > p.ny) throw std::runtime_error("xy-plane too large for the row-class split");
    int C = emax / p.nz;
    int w = C / P;
    if (w < 1) throw std::runtime_error("z-lines too long for the row-class count");
    if (w > p.nx) w = p.nx;
    g.P = P;
    g.Ly = p.ny / P;
    g.w = w;
    if (!p.force_generic && fast_z_supported(p.esize, p.nz, P, w)) p.fast_z = true;
    g.C = w * P;
    g.lgnx = lg2(p.nx);
    g.lgny = lg2(p.ny);
    g.lgnz = lg2(p.nz);
    g.lgP = lg2(P);
    g.lgLy = lg2(g.Ly);
    g.lgw = lg2(w);
    g.lgC = lg2(g.C);
    g.pitchXY = p.nx + (p.nx >= 16 ? 1 : 0);
    g.pitchZ = g.C;
    g.nblk_lg = lg2(p.nx / w);
    g.plane = (long long)p.nx * p.ny;
    g.batch = p.batch;
    g.lgzt = g.lgLy + g.nblk_lg;
    g.rstride = g.plane * p.nz;
    for (int i = 0; i < 6; ++i) g.box[i] = p.box[i];
    g.dx = (p.box[1] - p.box[0]) / p.nx;
    const size_t es = p.esize;
    if (xy_smem(g, (int)es) > 200 * 1024 || z_smem(g, (int)es) > 200 * 1024)
        throw std::runtime_error("tile exceeds the shared-memory budget");
    (void)maxv;
}

void build_twiddles(PlanState &p, std::vector<unsigned char> &host, int maxv)
{
    Geom &g = p.geom;
    int entries = 0;
    g.apx = make_axis(p.nx, maxv, entries);
    g.apy = make_axis(g.Ly, maxv, entries);
    g.apz = make_axis(p.nz, maxv, entries);
    g.cross_off = entries;
    entries += p.ny;
    g.fast_x_off = entries;
    entries += p.nx;
    g.fast_z_off = entries;
    entries += p.nz;
    g.fast_y_off = entries;
    entries += g.Ly;
    host.assign((size_t)entries * lift_size(p), 0);
    const AxisPlan *aps[3] = {&g.apx, &g.apy, &g.apz};
    for (int a = 0; a < 3; ++a) {
        const AxisPlan &ap = *aps[a];
        for (int s = 0; s < ap.nst; ++s) {
            if (ap.lgNs[s] == 0) continue;
            const long long M = (long long)ap.R[s] << ap.lgNs[s];
            for (long long e = 0; e < M; ++e) {
                double pp, u, sg;
                lift_rational(-2 * e, M, pp, u, sg);        // exp(-2 pi i e/M)
                put_any(p, host, (size_t)(ap.off[s] + e), pp, u, sg, 1.0);
            }
        }
    }
    const int full[4][2] = {{g.cross_off, p.ny}, {g.fast_x_off, p.nx}, {g.fast_z_off, p.nz},
                            {g.fast_y_off, g.Ly}};
    for (const auto &f : full) {
        for (long long e = 0; e < f[1]; ++e) {
            double pp, u, sg;
            lift_rational(-2 * e, f[1], pp, u, sg);          // exp(-2 pi i e/n)
            put_any(p, host, (size_t)(f[0] + e), pp, u, sg, 1.0);
        }
    }
}

// exp(-i (k^2/2) dt) per axis (real time) or exp(-(k^2/2) dt) (imaginary)
void build_kinetic(const PlanState &p, double dt, int imag, std::vector<unsigned char> &host)
{
    const int n[3] = {p.nx, p.ny, p.nz};
    host.assign((size_t)(p.nx + p.ny + p.nz) * lift_size(p), 0);
    size_t idx = 0;
    for (int a = 0; a < 3; ++a) {
        for (int m = 0; m < n[a]; ++m, ++idx) {
            const double k = wavenumber(m, n[a], p.box[2 * a], p.box[2 * a + 1]);
            const double th = 0.5 * k * k * dt;
            if (imag) {
                put_any(p, host, idx, 0.0, 0.0, 1.0, std::exp(-th));
            } else {
                double pp, u, sg;
                lift_angle(-th, pp, u, sg);
                put_any(p, host, idx, pp, u, sg, 1.0);
            }
        }
    }
}

void build_kinetic_xy(const PlanState &p, double dt, std::vector<unsigned char> &host)
{
    host.assign((size_t)p.nx * p.ny * lift_size(p), 0);
    for (int my = 0; my < p.ny; ++my) {
        const double ky = wavenumber(my, p.ny, p.box[2], p.box[3]);
        for (int mx = 0; mx < p.nx; ++mx) {
            const double kx = wavenumber(mx, p.nx, p.box[0], p.box[1]);
            double pp, u, sg;
            lift_angle(-0.5 * (kx * kx + ky * ky) * dt, pp, u, sg);
            put_any(p, host, (size_t)my * p.nx + mx, pp, u, sg, 1.0);
        }
    }
}

void build_k2h(const PlanState &p, std::vector<double> &host)
{
    const int n[3] = {p.nx, p.ny, p.nz};
    host.clear();
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < n[a]; ++m) {
            const double k = wavenumber(m, n[a], p.box[2 * a], p.box[2 * a + 1]);
            host.push_back(0.5 * k * k);
        }
}

// separable potential factors for tau = dt/2 (first block) and tau = dt
void build_separable(const PlanState &p, double dt, int imag, std::vector<unsigned char> &host)
{
    const size_t n = (size_t)(p.nx + p.ny + p.nz);
    host.assign(2 * n * lift_size(p), 0);
    for (int half = 0; half < 2; ++half) {
        const double tau = half == 0 ? 0.5 * dt : dt;
        for (size_t i = 0; i < n; ++i) {
            const double th = p.h_vsep[i] * tau;
            if (imag) {
                put_any(p, host, half * n + i, 0.0, 0.0, 1.0, std::exp(-th));
            } else {
                double pp, u, sg;
                lift_angle(-th, pp, u, sg);
                put_any(p, host, half * n + i, pp, u, sg, 1.0);
            }
        }
    }
}

// Cardinal basis of the natural cubic interpolating spline: B[m][i] is the
// spline through the unit data e_m evaluated at z[i].  Second derivatives
// from the tridiagonal continuity system (Thomas algorithm), zero at both
// ends; points outside the knots use the end interval's cubic.
void natural_spline_basis(const std::vector<double> &t, const std::vector<double> &z,
                          std::vector<double> &B)
{
    const int m = (int)t.size();
    B.assign((size_t)m * z.size(), 0.0);
    std::vector<double> h(m - 1);
    for (int i = 0; i + 1 < m; ++i) h[i] = t[i + 1] - t[i];
    std::vector<double> M(m), c(m), d(m);
    for (int col = 0; col < m; ++col) {
        // rhs for data y = e_col
        auto y = [&](int i) { return i == col ? 1.0 : 0.0; };
        std::fill(M.begin(), M.end(), 0.0);
        if (m > 2) {
            const int n = m - 2;   // unknowns M_1..M_{m-2}
            std::vector<double> a(n), b(n), cc(n), r(n);
            for (int k = 0; k < n; ++k) {
                const int i = k + 1;
                a[k] = h[i - 1];
                b[k] = 2.0 * (h[i - 1] + h[i]);
                cc[k] = h[i];
                r[k] = 6.0 * ((y(i + 1) - y(i)) / h[i] - (y(i) - y(i - 1)) / h[i - 1]);
            }
            for (int k = 1; k < n; ++k) {
                const double w = a[k] / b[k - 1];
                b[k] -= w * cc[k - 1];
                r[k] -= w * r[k - 1];
            }
            M[n] = r[n - 1] / b[n - 1];
            for (int k = n - 2; k >= 0; --k) M[k + 1] = (r[k] - cc[k] * M[k + 2]) / b[k];
        }
        for (size_t q = 0; q < z.size(); ++q) {
            int i = 0;
            while (i < m - 2 && z[q] >= t[i + 1]) ++i;
            const double aa = t[i + 1] - z[q], bb = z[q] - t[i], hh = h[i];
            B[(size_t)col * z.size() + q] = M[i] * aa * aa * aa / (6 * hh) +
                                            M[i + 1] * bb * bb * bb / (6 * hh) +
                                            (y(i) / hh - M[i] * hh / 6) * aa +
                                            (y(i + 1) / hh - M[i + 1] * hh / 6) * bb;
        }
    }
}

}  // namespace ctap
