// Host side of libfg21: errors, region construction (importance weighting,
// weighted-CDF partition, chromatic response precompute), model handles and
// the likelihood entry points of fg21.h.  All compute of the likelihood runs
// in the CUDA kernels of fg21_kernels.cu / fg21_tc.cu; nothing here evaluates
// a likelihood on the CPU.
#include <algorithm>
#include <queue>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fg21_internal.h"
#include "fg21_model.h"

namespace fg21 {

// ------------------------------------------------------------------ errors
static thread_local std::string tl_err;
static thread_local int64_t tl_invalid = 0;

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tl_err = buf;
    return code;
}

void set_invalid_count(int64_t n) { tl_invalid = n; }

int cuda_error(cudaError_t e, const char *what) {
    return set_error(FG21_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static void clear_error() { tl_err.clear(); }

// ---------------------------------------------------- region construction
// Importance of each pixel averaged over band and LST (Sec. 4.2):
//   W(pix,f,t) = num(pix,f,t) / sum_q num(q,f,t), w[pix] = (1/(F T)) sum_{f,t} W.
// num = T_sky D (beam), T_sky H (sky), H (horizon), 1 (uniform), with
// T_sky of eq. skyapproximation and the cos^p beam (H = above the horizon).
// Pixels are processed in fixed blocks so sums do not depend on the thread count.
namespace {

constexpr int64_t PIX_BLOCK = 1024;

struct Geometry {
    int64_t npix;
    int F, T;
    std::vector<double> logc;    // [npix][T] ln(z_t . v) or -inf below the horizon
    std::vector<double> lognu;   // [F] ln(nu_f / nu0)
};

void build_geometry(const fg21_sky *s, const fg21_obs *o, Geometry &g) {
    g.npix = s->npix;
    g.F = o->F;
    g.T = o->T;
    g.logc.resize((size_t)s->npix * o->T);
    g.lognu.resize(o->F);
    for (int f = 0; f < o->F; ++f) g.lognu[f] = std::log(o->nu[f] / o->nu0);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < s->npix; ++q) {
        const double *v = s->dirs + 3 * q;
        for (int t = 0; t < o->T; ++t) {
            const double *z = o->zenith + 3 * t;
            double c = v[0] * z[0] + v[1] * z[1] + v[2] * z[2];
            g.logc[(size_t)q * o->T + t] = c > 0.0 ? std::log(c) : -INFINITY;
        }
    }
}

inline double beam_at(const Geometry &g, const fg21_obs *o, int64_t q, int f, int t) {
    double lc = g.logc[(size_t)q * g.T + t];
    if (lc == -INFINITY) return 0.0;
    double p = o->beam_p[f];
    return 2.0 * (p + 1.0) * (p == 0.0 ? 1.0 : std::exp(p * lc));
}

inline double tsky_at(const fg21_sky *s, const fg21_obs *o, const Geometry &g, int64_t q, int f) {
    return (s->t230[q] - o->t_cmb) * std::exp(-s->beta[q] * g.lognu[f]) + o->t_cmb;
}

inline double importance_num(const fg21_sky *s, const fg21_obs *o, const Geometry &g, int weighting,
                             int64_t q, int f, int t, double tsky) {
    switch (weighting) {
        case FG21_WEIGHT_BEAM: return tsky * beam_at(g, o, q, f, t);
        case FG21_WEIGHT_SKY: return g.logc[(size_t)q * g.T + t] == -INFINITY ? 0.0 : tsky;
        case FG21_WEIGHT_HORIZON: return g.logc[(size_t)q * g.T + t] == -INFINITY ? 0.0 : 1.0;
        default: return 1.0;
    }
}

void importance(const fg21_sky *s, const fg21_obs *o, const Geometry &g, int weighting,
                std::vector<double> &w) {
    const int F = o->F, T = o->T;
    const int64_t npix = s->npix;
    const int64_t nblk = (npix + PIX_BLOCK - 1) / PIX_BLOCK;
    std::vector<double> part((size_t)nblk * F * T, 0.0);
#pragma omp parallel for schedule(dynamic)
    for (int64_t b = 0; b < nblk; ++b) {
        double *acc = &part[(size_t)b * F * T];
        for (int64_t q = b * PIX_BLOCK; q < std::min(npix, (b + 1) * PIX_BLOCK); ++q)
            for (int f = 0; f < F; ++f) {
                double ts = tsky_at(s, o, g, q, f);
                for (int t = 0; t < T; ++t) acc[f * T + t] += importance_num(s, o, g, weighting, q, f, t, ts);
            }
    }
    std::vector<double> den((size_t)F * T, 0.0);
    for (int64_t b = 0; b < nblk; ++b)
        for (int ft = 0; ft < F * T; ++ft) den[ft] += part[(size_t)b * F * T + ft];
    for (int ft = 0; ft < F * T; ++ft) den[ft] = den[ft] > 0.0 ? 1.0 / den[ft] : 0.0;
    w.assign(npix, 0.0);
    const double inv_ft = 1.0 / ((double)F * (double)T);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < npix; ++q) {
        double acc = 0.0;
        for (int f = 0; f < F; ++f) {
            double ts = tsky_at(s, o, g, q, f);
            for (int t = 0; t < T; ++t) acc += importance_num(s, o, g, weighting, q, f, t, ts) * den[f * T + t];
        }
        w[q] = acc * inv_ft;
    }
}

// Weighted CDF over a per-pixel field (eq. weighted_cdf; the field is beta
// for the spectral-index regions, the caller's field for amplitude regions):
// pixels sorted by (value, index), cum[k] = running importance.  C^-1(c) is
// the value of the first sorted pixel with cum >= c.
struct Cdf {
    std::vector<int64_t> order;
    std::vector<double> sorted_beta, cum;
    double inverse(double c) const {
        auto it = std::lower_bound(cum.begin(), cum.end(), c);
        if (it == cum.end()) return sorted_beta.back();
        return sorted_beta[it - cum.begin()];
    }
    // mass of (a, b] (or [a, b] if closed_below), summed in sorted order
    double mass(double a, double b, bool closed_below) const {
        auto lo = closed_below ? std::lower_bound(sorted_beta.begin(), sorted_beta.end(), a)
                               : std::upper_bound(sorted_beta.begin(), sorted_beta.end(), a);
        auto hi = std::upper_bound(sorted_beta.begin(), sorted_beta.end(), b);
        double m = 0.0;
        for (auto k = lo - sorted_beta.begin(); k < hi - sorted_beta.begin(); ++k) m += wsorted[k];
        return m;
    }
    std::vector<double> wsorted;
};

void make_cdf(int64_t n, const double *beta, const std::vector<double> &w, Cdf &c) {
    c.order.resize(n);
    for (int64_t k = 0; k < n; ++k) c.order[k] = k;
    std::sort(c.order.begin(), c.order.end(), [beta](int64_t i, int64_t j) {
        return beta[i] < beta[j] || (beta[i] == beta[j] && i < j);
    });
    c.sorted_beta.resize(n);
    c.wsorted.resize(n);
    c.cum.resize(n);
    double run = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        c.sorted_beta[k] = beta[c.order[k]];
        c.wsorted[k] = w[c.order[k]];
        run += c.wsorted[k];
        c.cum[k] = run;
    }
}

struct Region {
    double a, b, ca, cb;
    bool closed;   // recursive: the lowest region, closed below
};

// Algorithm 2 (recursive): repeatedly halve, at the beta midpoint, the region
// of largest importance mass; ties go to the lowest lower edge, then to the
// region created first.  A max-priority queue holds every region keyed by that
// rule, with each region's mass summed once when the region is made.
void split_recursive(const Cdf &c, int N, double bmin, double bmax, std::vector<Region> &R) {
    struct Key {
        double m, a;
        int idx;
    };
    // true when x is split after y
    auto later = [](const Key &x, const Key &y) {
        if (x.m != y.m) return x.m < y.m;
        if (x.a != y.a) return x.a > y.a;
        return x.idx > y.idx;
    };
    std::priority_queue<Key, std::vector<Key>, decltype(later)> q(later);
    R.assign(1, Region{bmin, bmax, 0.0, 0.0, true});
    q.push(Key{c.mass(bmin, bmax, true), bmin, 0});
    while ((int)R.size() < N) {
        const Key k = q.top();
        q.pop();
        Region &lo = R[k.idx];
        const double mid = 0.5 * (lo.a + lo.b);
        const Region up{mid, lo.b, 0.0, 0.0, false};
        lo.b = mid;
        q.push(Key{c.mass(lo.a, lo.b, lo.closed), lo.a, k.idx});
        R.push_back(up);
        q.push(Key{c.mass(up.a, up.b, false), up.a, (int)R.size() - 1});
    }
}

// Algorithm 1 (hierarchical): 2^floor(log2 N) base regions of equal target
// mass, then the widest base regions not yet bisected are bisected at their
// importance midpoints.  Unsplit base regions keep their widths, so the
// regions bisected are the first N - nb of the base regions in order of width
// (descending; ties to the lowest lower edge, then to the lower index).
void split_hierarchical(const Cdf &c, int N, double bmin, double bmax, std::vector<Region> &R) {
    int nb = 1;
    while (nb * 2 <= N) nb *= 2;
    R.clear();
    for (int j = 1; j <= nb; ++j) {
        const double cj = (double)j / nb;
        const double a = R.empty() ? bmin : R.back().b, ca = R.empty() ? 0.0 : R.back().cb;
        R.push_back(Region{a, j == nb ? bmax : c.inverse(cj), ca, cj, false});
    }
    std::vector<int> by_width(nb);
    for (int j = 0; j < nb; ++j) by_width[j] = j;
    std::stable_sort(by_width.begin(), by_width.end(), [&R](int x, int y) {
        const double wx = R[x].b - R[x].a, wy = R[y].b - R[y].a;
        return wx > wy || (wx == wy && R[x].a < R[y].a);
    });
    for (int k = 0; k < N - nb; ++k) {
        const Region r = R[by_width[k]];
        const double cm = 0.5 * (r.ca + r.cb), bm = c.inverse(cm);
        R[by_width[k]].b = bm;
        R[by_width[k]].cb = cm;
        R.push_back(Region{bm, r.b, cm, r.cb, false});
    }
}

// Algorithm 2 / Algorithm 1 / Sec. 4.1 splits -> ascending edges[N+1]: the
// regions tile [beta_min, beta_max], so the edges are beta_min and the sorted
// upper ends of the regions.
void split(const Cdf &c, int N, int scheme, std::vector<double> &edges) {
    const double bmin = c.sorted_beta.front(), bmax = c.sorted_beta.back();
    std::vector<Region> R;
    if (scheme == FG21_SCHEME_RECURSIVE) {
        split_recursive(c, N, bmin, bmax, R);
    } else if (scheme == FG21_SCHEME_HIERARCHICAL) {
        split_hierarchical(c, N, bmin, bmax, R);
    } else if (scheme == FG21_SCHEME_LINEAR) {
        for (int j = 0; j < N; ++j)
            R.push_back({j == 0 ? bmin : bmin + (bmax - bmin) * j / N,
                         j == N - 1 ? bmax : bmin + (bmax - bmin) * (j + 1) / N, 0, 0, false});
    } else {  // percentile: boundary j at the first sorted position with (k+1)/npix >= j/N
        const int64_t n = (int64_t)c.sorted_beta.size();
        double prev = bmin;
        for (int j = 1; j <= N; ++j) {
            int64_t k = ((int64_t)j * n + N - 1) / N - 1;
            double e = j == N ? bmax : c.sorted_beta[k];
            R.push_back({prev, e, 0, 0, false});
            prev = e;
        }
    }
    edges.resize(N + 1);
    edges[0] = bmin;
    for (int j = 0; j < N; ++j) edges[j + 1] = R[j].b;
    std::sort(edges.begin() + 1, edges.end());
}

// Chromatic response functions (Sec. 2.2 eq. chromatic_function with
// dOmega = 4 pi / Npix) and the beam normalisation B:
//   A[i,f,t] = (1/Npix) sum_{pix in i} (T230 - T_CMB) D,  B[f,t] = (1/Npix) sum_pix D.
// One channel per task, pixels in index order.
void precompute(const fg21_sky *s, const fg21_obs *o, const Geometry &g, const std::vector<int32_t> &lab,
                int N, std::vector<double> &A, std::vector<double> &B) {
    const int F = o->F, T = o->T;
    A.assign((size_t)N * F * T, 0.0);
    B.assign((size_t)F * T, 0.0);
    const double inv = 1.0 / (double)s->npix;
#pragma omp parallel
    {
        std::vector<double> acc((size_t)N * T), bacc(T);
#pragma omp for schedule(dynamic)
        for (int f = 0; f < F; ++f) {
            std::fill(acc.begin(), acc.end(), 0.0);
            std::fill(bacc.begin(), bacc.end(), 0.0);
            for (int64_t q = 0; q < s->npix; ++q) {
                double tmpl = s->t230[q] - o->t_cmb;
                double *ai = &acc[(size_t)lab[q] * T];
                for (int t = 0; t < T; ++t) {
                    double d = beam_at(g, o, q, f, t);
                    ai[t] += tmpl * d;
                    bacc[t] += d;
                }
            }
            for (int i = 0; i < N; ++i)
                for (int t = 0; t < T; ++t) A[((size_t)i * F + f) * T + t] = acc[(size_t)i * T + t] * inv;
            for (int t = 0; t < T; ++t) B[(size_t)f * T + t] = bacc[t] * inv;
        }
    }
}

int check_inputs(const fg21_sky *s, const fg21_obs *o) {
    if (!s || !o || !s->dirs || !s->t230 || !s->beta || !o->nu || !o->zenith || !o->beam_p)
        return set_error(FG21_E_ARG, "NULL sky/obs array");
    if (s->npix <= 0 || o->F <= 0 || o->T <= 0) return set_error(FG21_E_ARG, "npix, F and T must be > 0");
    if (!(o->nu0 > 0.0) || !std::isfinite(o->t_cmb)) return set_error(FG21_E_ARG, "nu0 must be > 0, t_cmb finite");
    for (int f = 0; f < o->F; ++f) {
        if (!(o->nu[f] > 0.0) || !std::isfinite(o->nu[f])) return set_error(FG21_E_ARG, "nu[%d] must be > 0", f);
        if (!(o->beam_p[f] >= 0.0) || !std::isfinite(o->beam_p[f]))
            return set_error(FG21_E_ARG, "beam_p[%d] must be >= 0", f);
    }
    for (int t = 0; t < o->T; ++t) {
        const double *z = o->zenith + 3 * t;
        double n = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
        if (!(std::fabs(n - 1.0) < 2e-6)) return set_error(FG21_E_ARG, "zenith[%d] is not a unit vector", t);
    }
    for (int64_t q = 0; q < s->npix; ++q) {
        const double *v = s->dirs + 3 * q;
        double n = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (!(std::fabs(n - 1.0) < 2e-6)) return set_error(FG21_E_ARG, "dirs[%lld] is not a unit vector", (long long)q);
        if (!std::isfinite(s->t230[q]) || !std::isfinite(s->beta[q]))
            return set_error(FG21_E_ARG, "non-finite t230/beta at pixel %lld", (long long)q);
    }
    return FG21_OK;
}

}  // namespace

}  // namespace fg21

using namespace fg21;

// ================================================================= C ABI
extern "C" {

const char *fg21_last_error(void) { return tl_err.c_str(); }
int64_t fg21_last_invalid_count(void) { return tl_invalid; }
const char *fg21_version(void) { return "fg21 1.0 (sm_103a)"; }

int fg21_device_count(void) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // extern "C"

namespace fg21 {
namespace {
struct Built {
    std::vector<double> edges, edges_a, A, B;
    std::vector<int32_t> lab, lab_a;
    int Nb = 0, Na = 0;          // Na = 0: no amplitude regions
    int n_empty = 0;             // components without a pixel
};

int check_opts(const fg21_sky *sky, int N, int scheme, int weighting, const char *what) {
    if (N < 1 || N > FG21_MAX_REGIONS || (int64_t)N > sky->npix)
        return set_error(FG21_E_ARG, "%s n_regions=%d must be in [1, min(npix, %d)]", what, N, FG21_MAX_REGIONS);
    if (scheme < 0 || scheme > 3) return set_error(FG21_E_ARG, "%s: unknown scheme %d", what, scheme);
    if (weighting < 0 || weighting > 3) return set_error(FG21_E_ARG, "%s: unknown weighting %d", what, weighting);
    return FG21_OK;
}

// Split `field` into N regions by the CDF of the importance w and label the
// pixels: region j holds values in (edges[j], edges[j+1]] (the lowest closed
// below), found by comparing each value with the edges.
void partition_field(int64_t npix, const double *field, const std::vector<double> &w, int N, int scheme,
                     std::vector<double> &edges, std::vector<int32_t> &lab) {
    Cdf c;
    make_cdf(npix, field, w, c);
    split(c, N, scheme, edges);
    lab.resize(npix);
    for (int64_t q = 0; q < npix; ++q)
        lab[q] = (int32_t)(std::lower_bound(edges.begin() + 1, edges.begin() + N, field[q]) - (edges.begin() + 1));
}

// Spectral-index regions (opt), optionally amplitude regions (aopt), and the
// response functions of their intersections: component i * Nb + j.  With
// `device` the O(Npix F T) sums (importance weights, response functions) run
// on the current GPU (fg21_build.cu); the partition is the same host code.
int build_host(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *opt,
               const fg21_amplitude_opts *aopt, Built &out, bool device) {
    if (!opt) return set_error(FG21_E_ARG, "NULL opt");
    int rc = check_inputs(sky, obs);
    if (rc) return rc;
    const int Nb = opt->n_regions;
    rc = check_opts(sky, Nb, opt->scheme, opt->weighting, "spectral-index");
    if (rc) return rc;
    int Na = 0;
    if (aopt) {
        Na = aopt->n_regions;
        rc = check_opts(sky, Na, aopt->scheme, aopt->weighting, "amplitude");
        if (rc) return rc;
        if (!aopt->field) return set_error(FG21_E_ARG, "NULL amplitude field");
        for (int64_t q = 0; q < sky->npix; ++q)
            if (!std::isfinite(aopt->field[q]))
                return set_error(FG21_E_ARG, "non-finite amplitude field at pixel %lld", (long long)q);
        if ((int64_t)Na * Nb > FG21_MAX_REGIONS)
            return set_error(FG21_E_ARG, "Na * Nb = %d components above %d", Na * Nb, FG21_MAX_REGIONS);
    }
    const int N = std::max(Na, 1) * Nb;
    try {
        Geometry g;
        if (!device) build_geometry(sky, obs, g);
        auto weights = [&](int weighting, std::vector<double> &w) -> int {
            if (device) return device_importance(sky, obs, weighting, w, nullptr);
            importance(sky, obs, g, weighting, w);
            return FG21_OK;
        };
        std::vector<double> w;
        if ((rc = weights(opt->weighting, w))) return rc;
        partition_field(sky->npix, sky->beta, w, Nb, opt->scheme, out.edges, out.lab);
        std::vector<int32_t> comp = out.lab;
        if (Na) {
            std::vector<double> wa;
            if (aopt->weighting != opt->weighting && (rc = weights(aopt->weighting, wa))) return rc;
            partition_field(sky->npix, aopt->field, aopt->weighting != opt->weighting ? wa : w, Na, aopt->scheme,
                            out.edges_a, out.lab_a);
            for (int64_t q = 0; q < sky->npix; ++q) comp[q] = out.lab_a[q] * Nb + out.lab[q];
        }
        if (device) {
            if ((rc = device_precompute(sky, obs, comp, N, out.A, out.B))) return rc;
        } else {
            precompute(sky, obs, g, comp, N, out.A, out.B);
        }
        std::vector<int64_t> count(N, 0);
        for (int64_t q = 0; q < sky->npix; ++q) count[comp[q]]++;
        out.n_empty = 0;
        for (int i = 0; i < N; ++i) out.n_empty += count[i] == 0;
        out.Nb = Nb;
        out.Na = Na;
    } catch (const std::bad_alloc &) {
        return set_error(FG21_E_NOMEM, "host allocation failed while building regions");
    }
    return FG21_OK;
}

// The device model of a built partition.
int make_model(const fg21_sky *sky, const fg21_obs *obs, Built &b, fg21_model **out) {
    fg21_model *m = nullptr;
    try {
        m = new fg21_model();
    } catch (const std::bad_alloc &) {
        return set_error(FG21_E_NOMEM, "host allocation failed");
    }
    m->n_beta = b.Nb;
    m->n_alpha = b.Na;
    m->N = std::max(b.Na, 1) * b.Nb;
    m->F = obs->F;
    m->T = obs->T;
    m->npix = sky->npix;
    m->n_empty = b.n_empty;
    m->nu0 = obs->nu0;
    m->t_cmb = obs->t_cmb;
    m->nu.assign(obs->nu, obs->nu + obs->F);
    m->edges = b.edges;
    m->edges_alpha = b.edges_a;
    m->A = std::move(b.A);
    m->B = std::move(b.B);
    int rc = model_upload(m);
    if (rc) {
        fg21_model_destroy(m);
        return rc;
    }
    *out = m;
    return FG21_OK;
}
}  // namespace
}  // namespace fg21

extern "C" {

int fg21_build_regions_host(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *opt,
                            int32_t *labels_out, double *edges_out, double *A_out, double *B_out) {
    clear_error();
    Built b;
    int rc = build_host(sky, obs, opt, nullptr, b, false);
    if (rc) return rc;
    if (labels_out) std::memcpy(labels_out, b.lab.data(), sizeof(int32_t) * b.lab.size());
    if (edges_out) std::memcpy(edges_out, b.edges.data(), sizeof(double) * b.edges.size());
    if (A_out) std::memcpy(A_out, b.A.data(), sizeof(double) * b.A.size());
    if (B_out) std::memcpy(B_out, b.B.data(), sizeof(double) * b.B.size());
    return FG21_OK;
}

int fg21_build_regions(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *opt,
                       fg21_model **out, int32_t *labels_out, double *edges_out) {
    clear_error();
    if (!out) return set_error(FG21_E_ARG, "NULL out");
    *out = nullptr;
    Built b;
    int rc = build_host(sky, obs, opt, nullptr, b, true);
    if (rc) return rc;
    if (labels_out) std::memcpy(labels_out, b.lab.data(), sizeof(int32_t) * sky->npix);
    if (edges_out) std::memcpy(edges_out, b.edges.data(), sizeof(double) * b.edges.size());
    return make_model(sky, obs, b, out);
}

int fg21_build_regions_ab_host(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *beta_opt,
                               const fg21_amplitude_opts *alpha_opt, int32_t *beta_labels, double *beta_edges,
                               int32_t *alpha_labels, double *alpha_edges, double *K_out, double *B_out) {
    clear_error();
    if (!alpha_opt) return set_error(FG21_E_ARG, "NULL alpha_opt");
    Built b;
    int rc = build_host(sky, obs, beta_opt, alpha_opt, b, false);
    if (rc) return rc;
    if (beta_labels) std::memcpy(beta_labels, b.lab.data(), sizeof(int32_t) * b.lab.size());
    if (beta_edges) std::memcpy(beta_edges, b.edges.data(), sizeof(double) * b.edges.size());
    if (alpha_labels) std::memcpy(alpha_labels, b.lab_a.data(), sizeof(int32_t) * b.lab_a.size());
    if (alpha_edges) std::memcpy(alpha_edges, b.edges_a.data(), sizeof(double) * b.edges_a.size());
    if (K_out) std::memcpy(K_out, b.A.data(), sizeof(double) * b.A.size());
    if (B_out) std::memcpy(B_out, b.B.data(), sizeof(double) * b.B.size());
    return FG21_OK;
}

int fg21_build_regions_ab(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *beta_opt,
                          const fg21_amplitude_opts *alpha_opt, fg21_model **out, int32_t *beta_labels,
                          double *beta_edges, int32_t *alpha_labels, double *alpha_edges) {
    clear_error();
    if (!out) return set_error(FG21_E_ARG, "NULL out");
    *out = nullptr;
    if (!alpha_opt) return set_error(FG21_E_ARG, "NULL alpha_opt");
    Built b;
    int rc = build_host(sky, obs, beta_opt, alpha_opt, b, true);
    if (rc) return rc;
    if (beta_labels) std::memcpy(beta_labels, b.lab.data(), sizeof(int32_t) * b.lab.size());
    if (beta_edges) std::memcpy(beta_edges, b.edges.data(), sizeof(double) * b.edges.size());
    if (alpha_labels) std::memcpy(alpha_labels, b.lab_a.data(), sizeof(int32_t) * b.lab_a.size());
    if (alpha_edges) std::memcpy(alpha_edges, b.edges_a.data(), sizeof(double) * b.edges_a.size());
    return make_model(sky, obs, b, out);
}

int fg21_simulate_data(const fg21_sky *sky, const fg21_obs *obs, const double *t21, double sigma_noise,
                       const double *noise, double *data_out) {
    clear_error();
    int rc = check_inputs(sky, obs);
    if (rc) return rc;
    if (!t21 || !data_out) return set_error(FG21_E_ARG, "NULL t21/data_out");
    try {
        Geometry g;
        build_geometry(sky, obs, g);
        const int F = obs->F, T = obs->T;
        const double inv = 1.0 / (double)sky->npix;
#pragma omp parallel
        {
            std::vector<double> acc(T);
#pragma omp for schedule(dynamic)
            for (int f = 0; f < F; ++f) {
                std::fill(acc.begin(), acc.end(), 0.0);
                for (int64_t q = 0; q < sky->npix; ++q) {
                    double ts = tsky_at(sky, obs, g, q, f);
                    for (int t = 0; t < T; ++t) acc[t] += beam_at(g, obs, q, f, t) * ts;
                }
                double dnu = obs->nu[f] - t21[1];
                double tr = t21[0] * std::exp(-(dnu * dnu) / (2.0 * t21[2] * t21[2]));
                for (int t = 0; t < T; ++t)
                    data_out[(size_t)f * T + t] = acc[t] * inv + tr + (noise ? sigma_noise * noise[(size_t)f * T + t] : 0.0);
            }
        }
    } catch (const std::bad_alloc &) {
        return set_error(FG21_E_NOMEM, "host allocation failed in fg21_simulate_data");
    }
    return FG21_OK;
}

}  // extern "C"
