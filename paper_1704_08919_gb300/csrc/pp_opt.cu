// pp_opt.cu -- the local search of Sec. IV.A of arXiv 1704.08919 on the host:
// augmented Lagrangian L = -J - lambda C + C^2 / (2 mu) with BFGS inner
// minimisation and a strong-Wolfe line search, started from many points at once.
//
// The paper defers the inner algorithms to Nocedal & Wright, "Numerical
// Optimization": the line search is their Algorithm 3.5 with the zoom of
// Algorithm 3.6 (cubic interpolation, Eq. 3.59, safeguarded by bisection); BFGS
// is Algorithm 6.1 with the inverse update of Eq. 6.17 and the first-step
// scaling of Eq. 6.20.  The outer loop takes the paper's steps 1-4: lambda_0 = 0,
// mu_0 > 0, minimise L(lambda_l, mu_l) from the previous minimiser, then
// lambda_{l+1} = lambda_l - C / mu_l and mu_{l+1} = xi mu_l, until |C| <= ctol.
//
// Multistart (step 5) runs every start in lockstep: each start is a state
// machine that stops wherever it needs the objective, and one batched call
// evaluates all pending points -- on the GPU, one launch for the whole batch.
// Every decision of a start depends only on its own values, so each start takes
// exactly the iterates a sequential run would.
#include <math.h>

#include <algorithm>
#include <vector>

#include "pp_internal.cuh"

namespace {

constexpr double kC1 = 1e-4;       // sufficient decrease
constexpr double kC2 = 0.9;        // curvature (strong Wolfe)
constexpr int kLsMax = 20;         // bracketing iterations
constexpr int kZoomMax = 30;       // zoom iterations
constexpr double kAlphaMax = 1e3;  // largest trial step
constexpr double kGrow = 2.0;      // step growth while bracketing

double dot(const std::vector<double> &a, const std::vector<double> &b)
{
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i)
        s += a[i] * b[i];
    return s;
}

// Minimiser of the cubic through (a, fa, ga), (b, fb, gb); false if none.
bool cubic_min(double a, double fa, double ga, double b, double fb, double gb, double *out)
{
    if (a == b)
        return false;
    const double d1 = ga + gb - 3.0 * (fa - fb) / (a - b);
    const double disc = d1 * d1 - ga * gb;
    if (disc < 0.0)
        return false;
    const double d2 = copysign(sqrt(disc), b - a);
    const double den = gb - ga + 2.0 * d2;
    if (den == 0.0)
        return false;
    *out = b - (b - a) * (gb + d2 - d1) / den;
    return true;
}

// A point of the line: step, value, directional derivative and what the
// objective returned there (trial point, gradient of L, J and C).
struct Pt {
    double a = 0.0, f = 0.0, d = 0.0;
    bool has = false;
    std::vector<double> x, g;
    double J = 0.0, C = 0.0;
};

struct Start {
    enum Phase { NEED_INIT, BRACKET, ZOOM, DONE };
    int n = 0;
    Phase phase = NEED_INIT;
    std::vector<double> x, g, H, p, req;  // req: the point whose evaluation is pending
    double f = 0.0, J = 0.0, C = 0.0;
    double lam = 0.0, mu = 1.0;
    int outer = 0, k = 0, evals = 0, status = 1;
    bool first = true;
    // line search
    double f0 = 0.0, g0 = 0.0, a = 0.0;
    int it = 0;
    Pt prev, lo, hi;
};

struct Search {
    int n;
    const pp_al_options *o;

    void request(Start &s, double a)
    {
        s.a = a;
        for (int i = 0; i < n; ++i)
            s.req[i] = s.x[i] + a * s.p[i];
    }

    double zoom_point(const Pt &l, const Pt &h)
    {
        double a;
        const double left = std::min(l.a, h.a), right = std::max(l.a, h.a), w = right - left;
        if (!cubic_min(l.a, l.f, l.d, h.a, h.f, h.d, &a) || !isfinite(a) ||
            !(left + 0.1 * w <= a && a <= right - 0.1 * w))
            a = 0.5 * (l.a + h.a);
        return a;
    }

    // Top of a BFGS iteration: converged or out of iterations ends the inner
    // minimisation; otherwise a direction and the first trial step.
    void iterate(Start &s)
    {
        double gmax = 0.0;
        for (int i = 0; i < n; ++i)
            gmax = std::max(gmax, fabs(s.g[i]));
        if (s.k >= o->max_iter || gmax <= o->gtol) {
            finish_inner(s);
            return;
        }
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j)
                acc += s.H[(size_t)i * n + j] * s.g[j];
            s.p[i] = -acc;
        }
        double gp = dot(s.p, s.g);
        if (!(gp < 0.0)) {  // not a descent direction: restart from the gradient
            std::fill(s.H.begin(), s.H.end(), 0.0);
            for (int i = 0; i < n; ++i) {
                s.H[(size_t)i * n + i] = 1.0;
                s.p[i] = -s.g[i];
            }
            gp = dot(s.p, s.g);
        }
        const double alpha1 = s.first ? std::min(1.0, 1.0 / sqrt(dot(s.g, s.g))) : 1.0;
        s.f0 = s.f;
        s.g0 = gp;
        s.prev = Pt();
        s.prev.f = s.f0;
        s.prev.d = s.g0;
        s.it = 0;
        s.phase = Start::BRACKET;
        request(s, alpha1);
    }

    // The line search ended at point e (e.has false: no step at all).
    void end_search(Start &s, const Pt &e, bool ok)
    {
        if (!e.has) {
            finish_inner(s);
            return;
        }
        std::vector<double> sv(n), y(n), Hy(n);
        for (int i = 0; i < n; ++i) {
            sv[i] = e.x[i] - s.x[i];
            y[i] = e.g[i] - s.g[i];
        }
        const double ys = dot(y, sv);
        if (ys > 0.0) {
            if (s.first) {  // Eq. 6.20
                const double sc = ys / dot(y, y);
                std::fill(s.H.begin(), s.H.end(), 0.0);
                for (int i = 0; i < n; ++i)
                    s.H[(size_t)i * n + i] = sc;
            }
            const double rho = 1.0 / ys;
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int j = 0; j < n; ++j)
                    acc += s.H[(size_t)i * n + j] * y[j];
                Hy[i] = acc;
            }
            const double c = rho * rho * dot(y, Hy) + rho;
            for (int i = 0; i < n; ++i)  // Eq. 6.17
                for (int j = 0; j < n; ++j)
                    s.H[(size_t)i * n + j] =
                        s.H[(size_t)i * n + j] - rho * (sv[i] * Hy[j] + Hy[i] * sv[j]) + c * (sv[i] * sv[j]);
        }
        s.first = false;
        s.x = e.x;
        s.f = e.f;
        s.g = e.g;
        s.J = e.J;
        s.C = e.C;
        s.k += 1;
        if (!ok) {
            finish_inner(s);
            return;
        }
        iterate(s);
    }

    void start_zoom(Start &s, const Pt &l, const Pt &h)
    {
        s.lo = l;
        s.hi = h;
        s.it = 0;
        s.phase = Start::ZOOM;
        request(s, zoom_point(s.lo, s.hi));
    }

    // The inner minimisation of L(lambda, mu) is over: feasible ends the search,
    // otherwise the multiplier and penalty are updated (steps 3, 4).
    void finish_inner(Start &s)
    {
        if (fabs(s.C) <= o->ctol) {
            s.outer += 1;
            s.status = 0;
            s.phase = Start::DONE;
            return;
        }
        s.lam = s.lam - s.C / s.mu;
        s.mu = o->xi * s.mu;
        s.outer += 1;
        if (s.outer >= o->outer) {
            s.status = 1;
            s.phase = Start::DONE;
            return;
        }
        s.req = s.x;
        s.phase = Start::NEED_INIT;
    }

    // L and its gradient from the objective's J, grad J, C, grad C.
    double lagrangian(const Start &s, double J, const double *gJ, double C, const double *gC,
                      std::vector<double> &g)
    {
        const double t = s.lam - C / s.mu;
        for (int i = 0; i < n; ++i)
            g[i] = -gJ[i] - t * gC[i];
        return -J - s.lam * C + C * C / (2.0 * s.mu);
    }

    void feed(Start &s, double J, const double *gJ, double C, const double *gC)
    {
        s.evals += 1;
        std::vector<double> gl(n);
        const double fl = lagrangian(s, J, gJ, C, gC, gl);
        if (s.phase == Start::NEED_INIT) {
            s.x = s.req;
            s.f = fl;
            s.g = gl;
            s.J = J;
            s.C = C;
            bool finite = isfinite(fl);
            for (int i = 0; i < n; ++i)
                finite = finite && isfinite(gl[i]);
            if (!finite) {  // the objective is not defined here: this start ends
                s.outer += 1;
                s.status = 2;
                s.phase = Start::DONE;
                return;
            }
            std::fill(s.H.begin(), s.H.end(), 0.0);
            for (int i = 0; i < n; ++i)
                s.H[(size_t)i * n + i] = 1.0;
            s.first = true;
            s.k = 0;
            iterate(s);
            return;
        }
        Pt cur;
        cur.a = s.a;
        cur.f = fl;
        cur.d = dot(gl, s.p);
        cur.has = true;
        cur.x = s.req;
        cur.g = gl;
        cur.J = J;
        cur.C = C;
        // a non-finite value or slope counts as a failed decrease (the step is too long)
        const bool bad = !(isfinite(cur.f) && isfinite(cur.d));
        if (s.phase == Start::BRACKET) {
            if (bad || cur.f > s.f0 + kC1 * cur.a * s.g0 || (s.it > 0 && cur.f >= s.prev.f)) {
                start_zoom(s, s.prev, cur);
                return;
            }
            if (fabs(cur.d) <= -kC2 * s.g0) {
                end_search(s, cur, true);
                return;
            }
            if (cur.d >= 0.0) {
                start_zoom(s, cur, s.prev);
                return;
            }
            s.prev = cur;
            s.it += 1;
            if (s.it >= kLsMax) {
                end_search(s, s.prev, false);
                return;
            }
            request(s, std::min(kGrow * cur.a, kAlphaMax));
            return;
        }
        // ZOOM
        if (bad || cur.f > s.f0 + kC1 * cur.a * s.g0 || cur.f >= s.lo.f) {
            s.hi = cur;
        } else {
            if (fabs(cur.d) <= -kC2 * s.g0) {
                end_search(s, cur, true);
                return;
            }
            if (cur.d * (s.hi.a - s.lo.a) >= 0.0)
                s.hi = s.lo;
            s.lo = cur;
        }
        s.it += 1;
        if (s.it >= kZoomMax) {
            end_search(s, s.lo, false);
            return;
        }
        request(s, zoom_point(s.lo, s.hi));
    }
};

}  // namespace

extern "C" {

int pp_al_search(int32_t n, int32_t nstart, double *x, pp_objective_fn fn, void *ctx,
                 const pp_al_options *opt, double *J_out, double *C_out, double *lam_out,
                 int32_t *evals_out, int32_t *outer_out, int32_t *status_out)
{
    pp::clear_error();
    if (n < 1 || nstart < 1 || !x || !fn || !opt)
        return pp::fail(PP_ERR_INVALID_ARG, "need n >= 1, nstart >= 1, x, an objective and options");
    if (!(opt->mu0 > 0.0) || !(opt->xi > 0.0 && opt->xi < 1.0) || opt->outer < 1 || opt->max_iter < 0 ||
        !(opt->gtol >= 0.0) || !(opt->ctol >= 0.0))
        return pp::fail(PP_ERR_INVALID_ARG, "options need mu0 > 0, 0 < xi < 1, outer >= 1, max_iter >= 0, "
                                            "gtol >= 0 and ctol >= 0");
    Search S{n, opt};
    std::vector<Start> st(nstart);
    for (int s = 0; s < nstart; ++s) {
        Start &q = st[s];
        q.n = n;
        q.x.assign(x + (size_t)s * n, x + (size_t)(s + 1) * n);
        q.req = q.x;
        q.g.assign(n, 0.0);
        q.p.assign(n, 0.0);
        q.H.assign((size_t)n * n, 0.0);
        q.mu = opt->mu0;
    }
    std::vector<int> act;
    std::vector<double> bx, bJ, bgJ, bC, bgC;
    for (;;) {
        act.clear();
        for (int s = 0; s < nstart; ++s)
            if (st[s].phase != Start::DONE)
                act.push_back(s);
        if (act.empty())
            break;
        const int m = (int)act.size();
        bx.resize((size_t)m * n);
        bJ.resize(m);
        bC.resize(m);
        bgJ.resize((size_t)m * n);
        bgC.resize((size_t)m * n);
        for (int q = 0; q < m; ++q)
            std::copy(st[act[q]].req.begin(), st[act[q]].req.end(), bx.begin() + (size_t)q * n);
        const int rc = fn(ctx, m, bx.data(), bJ.data(), bgJ.data(), bC.data(), bgC.data());
        if (rc)
            return rc == PP_OK ? PP_ERR_INVALID_ARG : rc;
        for (int q = 0; q < m; ++q)
            S.feed(st[act[q]], bJ[q], bgJ.data() + (size_t)q * n, bC[q], bgC.data() + (size_t)q * n);
    }
    for (int s = 0; s < nstart; ++s) {
        std::copy(st[s].x.begin(), st[s].x.end(), x + (size_t)s * n);
        if (J_out)
            J_out[s] = st[s].J;
        if (C_out)
            C_out[s] = st[s].C;
        if (lam_out)
            lam_out[s] = st[s].lam;
        if (evals_out)
            evals_out[s] = st[s].evals;
        if (outer_out)
            outer_out[s] = st[s].outer;
        if (status_out)
            status_out[s] = st[s].status;
    }
    return PP_OK;
}

}  // extern "C"
