// ts_path.cu -- host-side path planning: the Hufnagel-Valley Cn^2 profile (S21), the Rytov variance
// of one interval of a sampled profile (S19), and the screen-placement routine of Sec. 2.4 that turns
// a Cn^2 profile into the per-interval dz[] / Cn^2[] the split-step passes consume.
//
// The profile is piecewise linear between its samples (constant beyond the ends).  On a linear piece
// Cn^2 = a + b z the S19 integral has a closed form: with u = 1 - z / dz,
//   int (a + b z) (1 - z/dz)^(5/3) dz = dz [ (a + b dz) u^(8/3) / (8/3) - b dz u^(11/3) / (11/3) ]
// evaluated between the piece's ends (with a sign from dz = -dz du), so interval variances are exact
// up to rounding, with no quadrature.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ts_internal.h"

namespace ts {

namespace {

struct Profile {
    const double* z;
    const double* c;
    int n;
    double at(double x) const
    {
        if (x <= z[0]) return c[0];
        if (x >= z[n - 1]) return c[n - 1];
        const int i = (int)(std::upper_bound(z, z + n, x) - z) - 1;
        const double t = (x - z[i]) / (z[i + 1] - z[i]);
        return c[i] + t * (c[i + 1] - c[i]);
    }
};

// F(u) = (a + b dz) u^(8/3) * 3/8 - b dz u^(11/3) * 3/11, the antiderivative in u (times -1/dz)
double piece_primitive(double a, double b, double dz, double u)
{
    const double u83 = std::pow(u, 8.0 / 3.0), u113 = u83 * u;
    return (a + b * dz) * u83 * (3.0 / 8.0) - b * dz * u113 * (3.0 / 11.0);
}

// int_{z0}^{z1} Cn2(z) (1 - (z - z0)/(z1 - z0))^(5/3) dz over the piecewise-linear profile
double weighted_integral(const Profile& p, double z0, double z1)
{
    const double dz = z1 - z0;
    if (!(dz > 0.0)) return 0.0;
    // breakpoints inside (z0, z1)
    std::vector<double> br{z0};
    for (int i = 0; i < p.n; ++i)
        if (p.z[i] > z0 && p.z[i] < z1) br.push_back(p.z[i]);
    br.push_back(z1);
    double sum = 0.0;
    for (size_t k = 0; k + 1 < br.size(); ++k) {
        const double za = br[k], zb = br[k + 1];
        const double ca = p.at(za), cb = p.at(zb);
        // Cn2 = a + b (z - z0) on [za, zb]
        const double b = (cb - ca) / (zb - za);
        const double a = ca - b * (za - z0);
        const double ua = 1.0 - (za - z0) / dz, ub = 1.0 - (zb - z0) / dz;
        sum += dz * (piece_primitive(a, b, dz, ua) - piece_primitive(a, b, dz, ub));
    }
    return sum;
}

double interval_rytov(const Profile& p, double k, double z0, double z1)
{
    const double dz = z1 - z0;
    if (!(dz > 0.0)) return 0.0;
    return 3.27 * std::pow(k, 7.0 / 6.0) * std::pow(dz, 5.0 / 6.0) * weighted_integral(p, z0, z1);
}

// int_{z0}^{z1} Cn2(z) dz (exact for the piecewise-linear profile)
double plain_integral(const Profile& p, double z0, double z1)
{
    std::vector<double> br{z0};
    for (int i = 0; i < p.n; ++i)
        if (p.z[i] > z0 && p.z[i] < z1) br.push_back(p.z[i]);
    br.push_back(z1);
    double s = 0.0;
    for (size_t k = 0; k + 1 < br.size(); ++k) s += 0.5 * (p.at(br[k]) + p.at(br[k + 1])) * (br[k + 1] - br[k]);
    return s;
}

// the length d in (0, zmax - z0] at which the interval [z0, z0 + d] reaches the Rytov limit: the
// variance grows monotonically with d for a non-negative profile; bracketing by doubling, then
// regula falsi on log(sigma^2) against log(d) (S19 goes as d^(11/6) for a slowly varying profile,
// so the fit is close to linear there)
double length_to_limit(const Profile& p, double k, double z0, double zmax, double limit)
{
    if (interval_rytov(p, k, z0, zmax) <= limit) return zmax - z0;
    double lo = 0.0, hi = zmax - z0;
    double d = std::min(hi, 1.0);
    while (d < hi && interval_rytov(p, k, z0, z0 + d) < limit) {
        lo = d;
        d *= 2.0;
    }
    hi = std::min(d, hi);
    for (int it = 0; it < 200 && hi - lo > 1e-9 * (1.0 + hi); ++it) {
        double mid;
        if (lo > 0.0) {
            const double fl = std::log(interval_rytov(p, k, z0, z0 + lo) / limit);
            const double fh = std::log(interval_rytov(p, k, z0, z0 + hi) / limit);
            const double ll = std::log(lo), lh = std::log(hi);
            mid = (fh != fl) ? std::exp(ll - fl * (lh - ll) / (fh - fl)) : 0.5 * (lo + hi);
            if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
        } else {
            mid = 0.5 * (lo + hi);
        }
        if (interval_rytov(p, k, z0, z0 + mid) < limit) lo = mid;
        else hi = mid;
    }
    return lo > 0.0 ? lo : hi;
}

}  // namespace

}  // namespace ts

using ts::Profile;

extern "C" ts_status ts_cn2_hufnagel_valley(const double* h, int n, double V, double A, double* cn2)
{
    if (!h || !cn2 || n < 1 || !(V >= 0.0) || !(A >= 0.0)) {
        ts::set_error("ts_cn2_hufnagel_valley: need h, cn2, n >= 1, V >= 0, A >= 0");
        return TS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
        const double z = h[i];
        if (!(z >= 0.0)) {
            ts::set_error("ts_cn2_hufnagel_valley: heights must be >= 0");
            return TS_ERR_INVALID_ARG;
        }
        cn2[i] = 0.00594 * (V / 27.0) * (V / 27.0) * std::pow(1e-5 * z, 10.0) * std::exp(-z / 1000.0) +
                 2.7e-16 * std::exp(-z / 1500.0) + A * std::exp(-z / 100.0);
    }
    return TS_OK;
}

static ts_status check_profile(const double* z, const double* c, int n, const char* who)
{
    if (!z || !c || n < 1) {
        ts::set_error(std::string(who) + ": need a profile of n >= 1 samples");
        return TS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
        if (!(c[i] >= 0.0) || !std::isfinite(c[i]) || !std::isfinite(z[i]) || (i > 0 && !(z[i] > z[i - 1]))) {
            ts::set_error(std::string(who) + ": profile heights must increase and Cn^2 be finite and >= 0");
            return TS_ERR_INVALID_ARG;
        }
    }
    return TS_OK;
}

extern "C" ts_status ts_rytov_interval(const double* prof_z, const double* prof_cn2, int n_prof, double lambda,
                                       double z0, double z1, double* sigma2)
{
    ts_status st = check_profile(prof_z, prof_cn2, n_prof, "ts_rytov_interval");
    if (st != TS_OK) return st;
    if (!sigma2 || !(lambda > 0.0) || !(z1 >= z0)) {
        ts::set_error("ts_rytov_interval: need sigma2, lambda > 0 and z1 >= z0");
        return TS_ERR_INVALID_ARG;
    }
    const Profile p{prof_z, prof_cn2, n_prof};
    *sigma2 = ts::interval_rytov(p, 2.0 * M_PI / lambda, z0, z1);
    return TS_OK;
}

extern "C" ts_status ts_place_screens(const double* prof_z, const double* prof_cn2, int n_prof, const ts_medium* medium,
                                      const ts_grid* grid, double L, const double* init_bounds, int n_init,
                                      double rytov_limit, int max_screens, double* dz_out, double* cn2_out,
                                      double* rytov_out, int* n_out)
{
    ts_status st = check_profile(prof_z, prof_cn2, n_prof, "ts_place_screens");
    if (st != TS_OK) return st;
    if (!medium || !grid || !dz_out || !cn2_out || !n_out || !(L > 0.0) || !(rytov_limit > 0.0) || max_screens < 1 ||
        n_init < 0 || (n_init > 0 && !init_bounds)) {
        ts::set_error("ts_place_screens: need medium, grid, outputs, L > 0, rytov_limit > 0, max_screens >= 1");
        return TS_ERR_INVALID_ARG;
    }
    if (!(medium->lambda > 0.0)) {
        ts::set_error("ts_place_screens: lambda must be > 0");
        return TS_ERR_INVALID_ARG;
    }
    const Profile p{prof_z, prof_cn2, n_prof};
    const double n0 = medium->n0 > 0.0 ? medium->n0 : 1.0;
    const double k = 2.0 * M_PI * n0 / medium->lambda;
    const double dz_max = ts_max_step(medium, grid);
    if (!(dz_max > 0.0)) {
        ts::set_error("ts_place_screens: the grid has no valid Eq. 7 step limit");
        return TS_ERR_INVALID_ARG;
    }
    // 1. the user's intervals (boundaries strictly inside (0, L)), or one interval [0, L]
    std::vector<double> b{0.0};
    for (int i = 0; i < n_init; ++i)
        if (init_bounds[i] > b.back() && init_bounds[i] < L) b.push_back(init_bounds[i]);
    b.push_back(L);
    // 2. split intervals above the Rytov limit at their midpoints
    for (size_t i = 0; i + 1 < b.size();) {
        if (ts::interval_rytov(p, k, b[i], b[i + 1]) > rytov_limit && b[i + 1] - b[i] > 1e-6 * L) {
            b.insert(b.begin() + i + 1, 0.5 * (b[i] + b[i + 1]));
            if (b.size() > 1u << 20) break;
        } else {
            ++i;
        }
    }
    // 3. merge neighbours while the merged interval stays within the limit
    for (size_t i = 0; i + 2 < b.size();) {
        if (ts::interval_rytov(p, k, b[i], b[i + 2]) <= rytov_limit) b.erase(b.begin() + i + 1);
        else ++i;
    }
    // 4. final placement: each interval extended until it reaches the Rytov limit (linear fit of
    //    log sigma^2 against log dz between bracketing lengths)
    std::vector<double> f{0.0};
    while (f.back() < L * (1.0 - 1e-12)) {
        const double d = ts::length_to_limit(p, k, f.back(), L, rytov_limit);
        f.push_back(std::min(L, f.back() + std::max(d, 1e-9 * L)));
        if (f.size() > (size_t)max_screens + 2) break;  // already too many: reported below
    }
    f.back() = L;
    // keep whichever of the rough (2-3) and fitted (4) placements has fewer intervals
    std::vector<double>& best = (f.size() <= b.size()) ? f : b;
    // 5. split intervals longer than the Eq. 7 limit into equal parts
    std::vector<double> out{0.0};
    for (size_t i = 0; i + 1 < best.size(); ++i) {
        const double len = best[i + 1] - best[i];
        const int parts = std::max(1, (int)std::ceil(len / dz_max * (1.0 - 1e-12)));
        for (int j = 1; j <= parts; ++j) out.push_back(best[i] + len * j / parts);
    }
    const int n = (int)out.size() - 1;
    *n_out = n;
    if (n > max_screens) {
        ts::set_error("ts_place_screens: the placement needs " + std::to_string(n) + " screens, more than max_screens");
        return TS_ERR_WORKSPACE;
    }
    for (int i = 0; i < n; ++i) {
        const double dz = out[i + 1] - out[i];
        dz_out[i] = dz;
        cn2_out[i] = ts::plain_integral(p, out[i], out[i + 1]) / dz;  // path-integrated strength (S18) / dz
        if (rytov_out) rytov_out[i] = ts::interval_rytov(p, k, out[i], out[i + 1]);
    }
    return TS_OK;
}
