// Host side of the sources either side of the particle loop (Secs. 5.2, 5.3): the static
// gun field from the electrode potentials, and the table of the emission line.
#include <algorithm>
#include <cmath>

#include "pic_internal.h"

namespace pic {

// The static potential's system: for E = -grad phi, whose Whitney-1 edge values are
// phi(tail) - phi(head), the discrete Gauss law reads D_div star_eps D_div^T phi = Q (zero
// without space charge).  Because grad maps the Whitney-0 hats onto Whitney-1
// forms exactly, that matrix is the rho-weighted stiffness eps0 int rho grad(l_k).grad(l_l)
// over each triangle (rho linear: its mean times the area), assembled here per triangle.
// Held nodes keep their potential; the others solve the system (conjugate gradients,
// Jacobi preconditioner, relative residual 1e-13).
static pic_status solve_static(const HostMesh &m, const std::vector<uint8_t> &held,
                               const double *charge, std::vector<double> &phi) {
    const int64_t N0 = m.N0;
    std::vector<std::vector<std::pair<int32_t, double>>> rows(N0);
    for (int64_t t = 0; t < m.N2; t++) {
        const int32_t *n3 = &m.tri[3 * t];
        const double rbar = (m.zr[2 * n3[0] + 1] + m.zr[2 * n3[1] + 1] + m.zr[2 * n3[2] + 1]) / 3.0;
        const double w = m.units.eps0 * rbar * m.area[t];
        const double *g = &m.grad[6 * t];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                rows[n3[a]].push_back({n3[b], w * (g[2 * a] * g[2 * b] + g[2 * a + 1] * g[2 * b + 1])});
    }
    std::vector<int64_t> ptr(N0 + 1, 0);
    std::vector<int32_t> idx;
    std::vector<double> val;
    for (int64_t k = 0; k < N0; k++) {
        auto &r = rows[k];
        std::sort(r.begin(), r.end());
        for (size_t q = 0; q < r.size(); q++) {
            if ((int64_t)idx.size() > ptr[k] && idx.back() == r[q].first)
                val.back() += r[q].second;   // same column as the row's last entry
            else {
                idx.push_back(r[q].first);
                val.push_back(r[q].second);
            }
        }
        ptr[k + 1] = (int64_t)idx.size();
        std::vector<std::pair<int32_t, double>>().swap(r);
    }
    auto apply = [&](const std::vector<double> &x, std::vector<double> &y) {
        for (int64_t k = 0; k < N0; k++) {
            double s = 0.0;
            if (!held[k])
                for (int64_t q = ptr[k]; q < ptr[k + 1]; q++)
                    if (!held[idx[q]]) s += val[q] * x[idx[q]];
            y[k] = s;
        }
    };
    // right-hand side: the node charge minus the held potentials' coupling
    std::vector<double> b(N0, 0.0), diag(N0, 1.0);
    for (int64_t k = 0; k < N0; k++) {
        if (held[k]) continue;
        double s = charge ? charge[k] : 0.0;
        for (int64_t q = ptr[k]; q < ptr[k + 1]; q++) {
            if (held[idx[q]]) s -= val[q] * phi[idx[q]];
            if (idx[q] == k) diag[k] = val[q];
        }
        b[k] = s;
        if (!(diag[k] > 0.0)) {
            set_error("pic_static_potential: node %lld is not coupled to the mesh", (long long)k);
            return PIC_ERR_MESH;
        }
    }
    std::vector<double> x(N0, 0.0), r = b, z(N0), p(N0), Ap(N0);
    for (int64_t k = 0; k < N0; k++) z[k] = held[k] ? 0.0 : r[k] / diag[k];
    p = z;
    double rz = 0.0, bn = 0.0;
    for (int64_t k = 0; k < N0; k++) {
        rz += r[k] * z[k];
        bn += b[k] * b[k];
    }
    bn = std::sqrt(bn);
    const int64_t max_it = 20 * N0 + 100;
    bool done = bn == 0.0;
    for (int64_t it = 0; it < max_it && !done; it++) {
        apply(p, Ap);
        double pAp = 0.0;
        for (int64_t k = 0; k < N0; k++) pAp += p[k] * Ap[k];
        if (!(pAp > 0.0)) break;
        const double alpha = rz / pAp;
        double rn = 0.0;
        for (int64_t k = 0; k < N0; k++) {
            x[k] += alpha * p[k];
            r[k] -= alpha * Ap[k];
            rn += r[k] * r[k];
        }
        if (std::sqrt(rn) <= 1e-13 * bn) {
            done = true;
            break;
        }
        double rz2 = 0.0;
        for (int64_t k = 0; k < N0; k++) {
            z[k] = held[k] ? 0.0 : r[k] / diag[k];
            rz2 += r[k] * z[k];
        }
        const double beta = rz2 / rz;
        rz = rz2;
        for (int64_t k = 0; k < N0; k++) p[k] = z[k] + beta * p[k];
    }
    if (!done) {
        set_error("pic_static_potential: conjugate gradients did not converge (is every part "
                  "of the mesh connected to a held node?)");
        return PIC_ERR_MESH;
    }
    for (int64_t k = 0; k < N0; k++)
        if (!held[k]) phi[k] = x[k];
    return PIC_OK;
}

bool build_emit_line(const HostMesh &m, double z0, double rho0, double rho1,
                     std::vector<double> &ra, std::vector<double> &rb, std::vector<double> &la,
                     std::vector<double> &lb, std::vector<int32_t> &tri) {
    struct Iv {
        double a, b;
        double la[3], lb[3];
        int32_t t;
    };
    std::vector<Iv> iv;
    for (int64_t t = 0; t < m.N2; t++) {
        const int32_t *n3 = &m.tri[3 * t];
        double z[3], r[3];
        for (int k = 0; k < 3; k++) {
            z[k] = m.zr[2 * n3[k]];
            r[k] = m.zr[2 * n3[k] + 1];
        }
        if (std::min({z[0], z[1], z[2]}) >= z0 || std::max({z[0], z[1], z[2]}) <= z0) continue;
        // the line crosses two edges (no node lies on it): the crossing points and their
        // barycentric coordinates
        double pr[2], pl[2][3];
        int np = 0;
        for (int k = 0; k < 3 && np < 2; k++) {
            const int i = (k + 1) % 3, j = (k + 2) % 3;
            if ((z[i] - z0) * (z[j] - z0) >= 0.0) continue;
            const double w = (z0 - z[i]) / (z[j] - z[i]);
            pr[np] = r[i] + w * (r[j] - r[i]);
            pl[np][k] = 0.0;
            pl[np][i] = 1.0 - w;
            pl[np][j] = w;
            np++;
        }
        if (np != 2) continue;
        const int lo = pr[0] <= pr[1] ? 0 : 1, hi = 1 - lo;
        Iv v;
        v.t = (int32_t)t;
        v.a = pr[lo];
        v.b = pr[hi];
        for (int k = 0; k < 3; k++) {
            v.la[k] = pl[lo][k];
            v.lb[k] = pl[hi][k];
        }
        // clip to [rho0, rho1]
        if (v.b <= rho0 || v.a >= rho1 || !(v.b > v.a)) continue;
        const double a2 = std::max(v.a, rho0), b2 = std::min(v.b, rho1);
        double na[3], nb[3];
        for (int k = 0; k < 3; k++) {
            na[k] = v.la[k] + (a2 - v.a) / (v.b - v.a) * (v.lb[k] - v.la[k]);
            nb[k] = v.la[k] + (b2 - v.a) / (v.b - v.a) * (v.lb[k] - v.la[k]);
        }
        v.a = a2;
        v.b = b2;
        std::copy(na, na + 3, v.la);
        std::copy(nb, nb + 3, v.lb);
        iv.push_back(v);
    }
    std::sort(iv.begin(), iv.end(), [](const Iv &x, const Iv &y) { return x.a < y.a; });
    if (iv.empty()) return false;
    const double tol = 1e-9 * std::max(rho1, 1e-300);
    if (iv.front().a > rho0 + tol || iv.back().b < rho1 - tol) return false;
    for (size_t k = 0; k + 1 < iv.size(); k++)
        if (std::fabs(iv[k].b - iv[k + 1].a) > tol) return false;   // a gap or an overlap
    ra.clear();
    rb.clear();
    la.clear();
    lb.clear();
    tri.clear();
    for (const Iv &v : iv) {
        ra.push_back(v.a);
        rb.push_back(v.b);
        tri.push_back(v.t);
        for (int k = 0; k < 3; k++) {
            la.push_back(v.la[k]);
            lb.push_back(v.lb[k]);
        }
    }
    return true;
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_static_potential(const pic_mesh *pm, int64_t n_held,
                                           const int32_t *held_nodes, const double *held_phi,
                                           const double *charge, double *phi_out,
                                           double *E_out) try {
    if (!pm || n_held <= 0 || !held_nodes || !held_phi) {
        set_error("pic_static_potential: bad argument");
        return PIC_ERR_ARG;
    }
    const HostMesh &m = pm->h;
    std::vector<uint8_t> held(m.N0, 0);
    std::vector<double> phi(m.N0, 0.0);
    for (int64_t k = 0; k < n_held; k++) {
        const int32_t n = held_nodes[k];
        if (n < 0 || n >= m.N0 || !std::isfinite(held_phi[k])) {
            set_error("pic_static_potential: held node %lld out of range or not finite", (long long)k);
            return PIC_ERR_ARG;
        }
        held[n] = 1;
        phi[n] = held_phi[k];
    }
    if (charge)
        for (int64_t k = 0; k < m.N0; k++)
            if (!std::isfinite(charge[k])) {
                set_error("pic_static_potential: node charge %lld is not finite", (long long)k);
                return PIC_ERR_ARG;
            }
    pic_status st = solve_static(m, held, charge, phi);
    if (st != PIC_OK) return st;
    if (phi_out) std::copy(phi.begin(), phi.end(), phi_out);
    if (E_out)
        for (int64_t e = 0; e < m.N1; e++)
            E_out[e] = phi[m.edge_nodes[2 * e]] - phi[m.edge_nodes[2 * e + 1]];
    return PIC_OK;
}
PIC_CATCH("pic_static_potential")
