// C ABI: ADAPT-VQE with every angle re-optimised (energy and adjoint
// gradient of the Taylor-5 product ansatz, BFGS, the outer loop).
#include "api_internal.h"
#include "dev.cuh"
#include "grad.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using namespace tq;
using namespace tq::api;

// ===================================================== ADAPT-VQE (re-optimised)

namespace {

// E(theta) and dE/dtheta of psi(theta) = U_n ... U_1 psi0 (Taylor-5 factors,
// no renormalisation): forward states phi_0 .. phi_n kept in scratch, the
// energy pass over phi_n (w = H psi), chi = w - E psi, then per factor from
// the last: the gradient dot, and chi <- U_j(-theta_j) chi.  `grad` (host)
// may be null; `psi_out` (device, D amplitudes) receives phi_n if not null.
double ansatz_energy_grad(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi0, int n, const int* ops,
                          const double* th, double* grad, void* psi_out, cudaStream_t s) {
    check_space(p, psi0);
    check_space(h, psi0);
    TQ_REQUIRE(h->prec == psi0->prec, "state and Hamiltonian precisions differ");
    TQ_REQUIRE(n >= 0, "n_ops < 0");
    for (int j = 0; j < n; ++j) {
        TQ_REQUIRE(ops[j] >= 0 && ops[j] < p->M, "pool index out of range");
        TQ_REQUIRE(std::isfinite(th[j]), "theta is not finite");
    }
    const int prec = psi0->prec;
    const long long D = psi0->D;
    const size_t vb = (size_t)D * elem_bytes(prec);
    double* part = prepare(c, D, p, p->nq);
    unsigned char* phis = static_cast<unsigned char*>(scratch(c, S_PHI, (size_t)(n + 1) * vb));
    void* chi = scratch(c, S_CHI, vb);
    double* gdev = static_cast<double*>(scratch(c, S_AG, (size_t)std::max(n, 1) * sizeof(double)));
    const int upt = c->pair_upt[prec];
    TQ_CUDA(cudaMemcpyAsync(phis, psi0->data, vb, cudaMemcpyDeviceToDevice, s));
    for (int j = 0; j < n; ++j) {
        unsigned char* dst = phis + (size_t)(j + 1) * vb;
        TQ_CUDA(cudaMemcpyAsync(dst, phis + (size_t)j * vb, vb, cudaMemcpyDeviceToDevice, s));
        launch_update(c, p, 1, prec, upt, dst, nullptr, nullptr, ops[j], th[j], nullptr, part, nullptr, nullptr, s);
    }
    tq_state last = *psi0;
    last.owned = 0;
    last.data = phis + (size_t)n * vb;
    run_energy(c, h, &last, part, s);
    if (grad) {
        launch(c, "residual", s, [&] { return launch_residual(static_cast<double2*>(c->scratch[S_W0]), last.data, chi, prec,
                                                              D, c->step, s); });
        for (int j = n - 1; j >= 0; --j) {
            const double t = th[j], t2 = t * t;
            const double c4 = 1.0 - t2 / 2.0 + t2 * t2 / 24.0, s4 = t * (1.0 - t2 / 6.0);
            launch(c, "ansatz_dot", s, [&] {
                return launch_ansatz_dot(p->view, ops[j], c4, s4, chi, phis + (size_t)j * vb, prec, D, part,
                                         c->tickets + 4, c->step, gdev + j, c->sm_count, s);
            });
            launch_update(c, p, 1, prec, upt, chi, nullptr, nullptr, ops[j], -t, nullptr, part, nullptr, nullptr, s);
        }
    }
    double E = 0.0;
    int status = 0;
    TQ_CUDA(cudaMemcpyAsync(&E, &c->step->energy, sizeof(double), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaMemcpyAsync(&status, &c->step->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (grad && n > 0) TQ_CUDA(cudaMemcpyAsync(grad, gdev, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (psi_out) TQ_CUDA(cudaMemcpyAsync(psi_out, last.data, vb, cudaMemcpyDeviceToDevice, s));
    TQ_CUDA(cudaStreamSynchronize(s));
    raise_status(c, status, s);
    return E;
}

// BFGS on f with gradient g: inverse-Hessian update, backtracking line
// search (Armijo, halving), restart along -g when the direction does not
// descend; stops when max |g_i| < gtol or after max_iter iterations.
// Returns f at the result; x is updated in place.
template <typename FG>
double bfgs(FG fg, std::vector<double>& x, double gtol, int max_iter, int* n_eval) {
    const size_t n = x.size();
    std::vector<double> g(n), gn(n), xn(n), d(n), sv(n), yv(n), Hy(n);
    std::vector<double> H(n * n, 0.0);
    for (size_t i = 0; i < n; ++i) H[i * n + i] = 1.0;
    double f = fg(x, g);
    int evals = 1;
    auto gmax = [](const std::vector<double>& v) {
        double m = 0.0;
        for (double e : v) m = std::max(m, std::fabs(e));
        return m;
    };
    for (int it = 0; it < max_iter && gmax(g) >= gtol; ++it) {
        double gd = 0.0;
        for (size_t i = 0; i < n; ++i) {
            double v = 0.0;
            for (size_t j = 0; j < n; ++j) v -= H[i * n + j] * g[j];
            d[i] = v;
            gd += v * g[i];
        }
        if (!(gd < 0.0)) {                         // not a descent direction: restart
            std::fill(H.begin(), H.end(), 0.0);
            for (size_t i = 0; i < n; ++i) H[i * n + i] = 1.0, d[i] = -g[i];
            gd = 0.0;
            for (size_t i = 0; i < n; ++i) gd -= g[i] * g[i];
        }
        double a = 1.0, fn = f;
        bool ok = false;
        for (int ls = 0; ls < 40; ++ls) {
            for (size_t i = 0; i < n; ++i) xn[i] = x[i] + a * d[i];
            fn = fg(xn, gn);
            ++evals;
            if (fn <= f + 1e-4 * a * gd) {
                ok = true;
                break;
            }
            a *= 0.5;
        }
        if (!ok) break;                            // no decrease along d: converged to rounding
        double sy = 0.0, yy = 0.0;
        for (size_t i = 0; i < n; ++i) {
            sv[i] = xn[i] - x[i];
            yv[i] = gn[i] - g[i];
            sy += sv[i] * yv[i];
            yy += yv[i] * yv[i];
        }
        if (sy > 1e-300) {
            if (it == 0) {                         // scale the first inverse Hessian
                std::fill(H.begin(), H.end(), 0.0);
                for (size_t i = 0; i < n; ++i) H[i * n + i] = sy / yy;
            }
            double yHy = 0.0;
            for (size_t i = 0; i < n; ++i) {
                double v = 0.0;
                for (size_t j = 0; j < n; ++j) v += H[i * n + j] * yv[j];
                Hy[i] = v;
                yHy += yv[i] * v;
            }
            const double rho = 1.0 / sy;
            for (size_t i = 0; i < n; ++i)
                for (size_t j = 0; j < n; ++j)
                    H[i * n + j] += -rho * (Hy[i] * sv[j] + sv[i] * Hy[j]) + (rho * rho * yHy + rho) * sv[i] * sv[j];
        }
        x = xn;
        g = gn;
        f = fn;
    }
    if (n_eval) *n_eval = evals;
    return f;
}

// The operator choice of the ADAPT step on host gradients (the tie rule of
// k_select): the lowest index within tau of max |g|.
int select_host(const std::vector<double>& g, int prec, double* gmax_out) {
    double gm = 0.0;
    for (double v : g) gm = std::max(gm, std::fabs(v));
    const double tau = prec == TQ_C128 ? 1e-9 * std::max(1.0, gm) : 1e-5;
    int k = 0;
    for (size_t i = 0; i < g.size(); ++i)
        if (std::fabs(g[i]) >= gm - tau) {
            k = (int)i;
            break;
        }
    *gmax_out = gm;
    return k;
}

}  // namespace

extern "C" int tq_ansatz_energy_grad(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi0, int n_ops,
                                     const int* ops, const double* thetas, double* E, double* grad, tq_state* psi_out,
                                     void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && h && p && psi0 && E, "null argument");
    TQ_REQUIRE(n_ops == 0 || (ops && thetas), "null argument");
    if (psi_out) {
        check_space(p, psi_out);
        TQ_REQUIRE(psi_out->prec == psi0->prec, "output state precision differs");
    }
    set_device(c);
    *E = ansatz_energy_grad(c, h, p, psi0, n_ops, ops, thetas, grad, psi_out ? psi_out->data : nullptr,
                            as_stream(stream));
    API_END
}

extern "C" int tq_adapt_vqe(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi0, double eps,
                            int max_ops, double gtol, int max_iter, int* n_ops, int* ops_out, double* thetas_out,
                            double* energies_out, tq_state* psi_out) {
    API_BEGIN
    TQ_REQUIRE(c && h && p && psi0 && n_ops && ops_out && thetas_out && energies_out, "null argument");
    TQ_REQUIRE(max_ops >= 0 && max_iter >= 0, "max_ops and max_iter must be >= 0");
    TQ_REQUIRE(std::isfinite(eps) && eps >= 0.0 && std::isfinite(gtol) && gtol > 0.0, "eps >= 0 and gtol > 0 required");
    check_space(p, psi0);
    check_space(h, psi0);
    set_device(c);
    cudaStream_t s = 0;
    const long long D = psi0->D;
    std::vector<int> ops;
    std::vector<double> th;
    std::vector<double> g(p->M);
    int count = 0;
    for (int it = 0; it < max_ops; ++it) {
        // psi(theta) and every pool gradient there
        void* work = scratch(c, S_STAGE, (size_t)D * elem_bytes(psi0->prec));
        ansatz_energy_grad(c, h, p, psi0, (int)ops.size(), ops.data(), th.data(), nullptr, work, s);
        tq_state cur = *psi0;
        cur.owned = 0;
        cur.data = work;
        double* gd = static_cast<double*>(scratch(c, S_G, (size_t)p->M * sizeof(double)));
        double* part = prepare(c, D, p, p->nq);
        run_gradients(c, h, p, &cur, gd, part, s);
        TQ_CUDA(cudaMemcpyAsync(g.data(), gd, (size_t)p->M * sizeof(double), cudaMemcpyDeviceToHost, s));
        TQ_CUDA(cudaStreamSynchronize(s));
        double gmax = 0.0;
        const int k = select_host(g, psi0->prec, &gmax);
        if (gmax < eps) break;
        ops.push_back(k);
        th.push_back(0.0);
        const double E = bfgs(
            [&](const std::vector<double>& x, std::vector<double>& gr) {
                return ansatz_energy_grad(c, h, p, psi0, (int)ops.size(), ops.data(), x.data(), gr.data(), nullptr, s);
            },
            th, gtol, max_iter, nullptr);
        ops_out[count] = k;
        energies_out[count] = E;
        ++count;
    }
    for (int j = 0; j < count; ++j) thetas_out[j] = th[j];
    *n_ops = count;
    if (psi_out) {
        check_space(p, psi_out);
        ansatz_energy_grad(c, h, p, psi0, count, ops.data(), th.data(), nullptr, psi_out->data, s);
    }
    API_END
}
