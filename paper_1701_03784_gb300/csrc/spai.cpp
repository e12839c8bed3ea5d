// Sparse approximate inverse of the Hodge matrix star_eps (Sec. 3.1) and the stable
// leapfrog step, host side, multithreaded over columns / rows.
#include <algorithm>
#include <cmath>
#include <thread>

#include "pic_internal.h"

namespace pic {

// min ||A x - b||_2 for a dense column-major A (rows >= cols) by Householder QR.
static void least_squares(std::vector<double> &A, int rows, int cols, std::vector<double> &b,
                          std::vector<double> &x) {
    for (int k = 0; k < cols; k++) {
        double *a = &A[(size_t)k * rows];
        double nrm = 0;
        for (int i = k; i < rows; i++) nrm += a[i] * a[i];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = a[k] > 0 ? -nrm : nrm;
        // v = a[k:] - alpha e_k, stored in place; H = I - 2 v v^T / (v^T v)
        a[k] -= alpha;
        double vtv = 0;
        for (int i = k; i < rows; i++) vtv += a[i] * a[i];
        for (int j = k + 1; j < cols; j++) {
            double *c = &A[(size_t)j * rows];
            double s = 0;
            for (int i = k; i < rows; i++) s += a[i] * c[i];
            s = 2.0 * s / vtv;
            for (int i = k; i < rows; i++) c[i] -= s * a[i];
        }
        double s = 0;
        for (int i = k; i < rows; i++) s += a[i] * b[i];
        s = 2.0 * s / vtv;
        for (int i = k; i < rows; i++) b[i] -= s * a[i];
        // R's diagonal entry; the reflector is no longer needed below row k
        a[k] = alpha;
    }
    x.assign(cols, 0.0);
    for (int k = cols - 1; k >= 0; k--) {
        double s = b[k];
        for (int j = k + 1; j < cols; j++) s -= A[(size_t)j * rows + k] * x[j];
        x[k] = s / A[(size_t)k * rows + k];
    }
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_spai_build(pic_mesh *pm, int32_t level, double drop_tol,
                                     double *dt_stable_out) try {
    if (!pm || level < 0 || level > 8 || !(drop_tol >= 0.0 && drop_tol < 1.0)) {
        set_error("pic_spai_build: bad argument");
        return PIC_ERR_ARG;
    }
    HostMesh &m = pm->h;
    const int64_t nf = (int64_t)m.free_edges.size();
    if (nf == 0) {
        set_error("pic_spai_build: no free edges");
        return PIC_ERR_MESH;
    }
    // edge adjacency through triangles (all edges, diagonal included)
    std::vector<int64_t> adj_ptr(m.N1 + 1, 0);
    std::vector<int32_t> adj;
    for (int64_t e = 0; e < m.N1; e++) {
        int32_t nb[6];
        int c = 0;
        for (int s = 0; s < 2; s++) {
            int32_t t = m.edge_face[2 * e + s];
            if (t < 0) continue;
            for (int k = 0; k < 3; k++) nb[c++] = m.tri_edge[3 * t + k];
        }
        std::sort(nb, nb + c);
        c = (int)(std::unique(nb, nb + c) - nb);
        adj.insert(adj.end(), nb, nb + c);
        adj_ptr[e + 1] = (int64_t)adj.size();
    }
    // free part of star_eps, column access (it is symmetric: rows of column j = row j)
    std::vector<std::vector<std::pair<int32_t, double>>> cols_out(nf);
    std::vector<uint8_t> bad(1, 0);
    parallel_for(nf, [&](int64_t j0, int64_t j1) {
        std::vector<int32_t> mark(m.N1, -1), S, Snext, R;
        std::vector<int32_t> rowpos(m.N1, -1);
        std::vector<double> A, b, x;
        for (int64_t j = j0; j < j1; j++) {
            int32_t ej = m.free_edges[j];
            // level-k pattern over all edges, then restricted to free edges
            S.assign(1, ej);
            mark[ej] = (int32_t)j;
            size_t lo = 0;
            for (int lv = 0; lv < level; lv++) {
                size_t hi = S.size();
                for (size_t q = lo; q < hi; q++) {
                    int32_t e = S[q];
                    for (int64_t k = adj_ptr[e]; k < adj_ptr[e + 1]; k++)
                        if (mark[adj[k]] != (int32_t)j) {
                            mark[adj[k]] = (int32_t)j;
                            S.push_back(adj[k]);
                        }
                }
                lo = hi;
            }
            Snext.clear();
            for (int32_t e : S)
                if (m.free_of_edge[e] >= 0) Snext.push_back(e);
            std::sort(Snext.begin(), Snext.end());
            // rows touched by the pattern's columns (free rows only)
            R.clear();
            for (int32_t e : Snext)
                for (int64_t k = m.eps_ptr[e]; k < m.eps_ptr[e + 1]; k++) {
                    int32_t r = m.eps_idx[k];
                    if (m.free_of_edge[r] >= 0 && rowpos[r] < 0) {
                        rowpos[r] = 0;
                        R.push_back(r);
                    }
                }
            std::sort(R.begin(), R.end());
            for (size_t i = 0; i < R.size(); i++) rowpos[R[i]] = (int32_t)i;
            int rows = (int)R.size(), ncol = (int)Snext.size();
            A.assign((size_t)rows * ncol, 0.0);
            for (int c = 0; c < ncol; c++) {
                int32_t e = Snext[c];
                for (int64_t k = m.eps_ptr[e]; k < m.eps_ptr[e + 1]; k++) {
                    int32_t r = m.eps_idx[k];
                    if (m.free_of_edge[r] >= 0) A[(size_t)c * rows + rowpos[r]] = m.eps_val[k];
                }
            }
            b.assign(rows, 0.0);
            b[rowpos[ej]] = 1.0;
            for (int32_t r : R) rowpos[r] = -1;
            least_squares(A, rows, ncol, b, x);
            double mx = 0;
            for (double v : x) mx = std::max(mx, std::fabs(v));
            if (!(mx > 0) || !std::isfinite(mx)) {
                bad[0] = 1;
                continue;
            }
            auto &col = cols_out[j];
            col.clear();
            for (int c = 0; c < ncol; c++)
                if (std::fabs(x[c]) >= drop_tol * mx)
                    col.push_back({m.free_of_edge[Snext[c]], x[c]});
        }
    });
    if (bad[0]) {
        set_error("pic_spai_build: a least-squares column failed");
        return PIC_ERR_MESH;
    }
    // M <- (M + M^T) / 2, as triplets sorted by (row, col)
    std::vector<std::pair<uint64_t, double>> trip;
    for (int64_t j = 0; j < nf; j++)
        for (auto &rv : cols_out[j]) {
            trip.push_back({(uint64_t)rv.first * (uint64_t)nf + (uint64_t)j, 0.5 * rv.second});
            trip.push_back({(uint64_t)j * (uint64_t)nf + (uint64_t)rv.first, 0.5 * rv.second});
        }
    std::sort(trip.begin(), trip.end(),
              [](const auto &x, const auto &y) { return x.first < y.first; });
    m.M_ptr.assign(nf + 1, 0);
    m.M_idx.clear();
    m.M_val.clear();
    for (size_t i = 0; i < trip.size();) {
        size_t j = i;
        double v = 0;
        while (j < trip.size() && trip[j].first == trip[i].first) v += trip[j++].second;
        m.M_idx.push_back((int32_t)(trip[i].first % (uint64_t)nf));
        m.M_val.push_back(v);
        m.M_ptr[trip[i].first / (uint64_t)nf + 1]++;
        i = j;
    }
    for (int64_t r = 0; r < nf; r++) m.M_ptr[r + 1] += m.M_ptr[r];

    // power iteration on M K, K = D_curl^T star_mu^-1 D_curl over free edges
    std::vector<double> x(nf), y(nf), kx(nf), tf(m.N2);
    double nrm = 0;
    for (int64_t i = 0; i < nf; i++) {
        x[i] = 1.0 + 0.5 * std::sin((double)(i + 1));
        nrm += x[i] * x[i];
    }
    nrm = std::sqrt(nrm);
    for (auto &v : x) v /= nrm;
    double lam = 0;
    for (int it = 0; it < 500; it++) {
        parallel_for(m.N2, [&](int64_t a, int64_t b) {
            for (int64_t t = a; t < b; t++) {
                double s = 0;
                for (int k = 0; k < 3; k++) {
                    int32_t e = m.tri_edge[3 * t + k];
                    int32_t f = m.free_of_edge[e];
                    if (f < 0) continue;
                    int32_t na = m.tri[3 * t + (k + 1) % 3], nb = m.tri[3 * t + (k + 2) % 3];
                    s += (na < nb ? 1.0 : -1.0) * x[f];
                }
                tf[t] = m.mu_inv[t] * s;
            }
        });
        parallel_for(nf, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; i++) {
                int32_t e = m.free_edges[i];
                double s = 0;
                for (int q = 0; q < 2; q++) {
                    int32_t t = m.edge_face[2 * e + q];
                    if (t >= 0) s += m.edge_face_sign[2 * e + q] * tf[t];
                }
                kx[i] = s;
            }
        });
        parallel_for(nf, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; i++) {
                double s = 0;
                for (int64_t k = m.M_ptr[i]; k < m.M_ptr[i + 1]; k++) s += m.M_val[k] * kx[m.M_idx[k]];
                y[i] = s;
            }
        });
        double n2 = 0;
        for (double v : y) n2 += v * v;
        lam = std::sqrt(n2);
        if (!(lam > 0) || !std::isfinite(lam)) {
            set_error("pic_spai_build: power iteration failed");
            return PIC_ERR_MESH;
        }
        for (int64_t i = 0; i < nf; i++) x[i] = y[i] / lam;
    }
    m.lambda_max = lam;
    m.dt_stable = 2.0 / std::sqrt(lam);
    m.have_spai = true;
    if (dt_stable_out) *dt_stable_out = m.dt_stable;
    return PIC_OK;
}
PIC_CATCH("pic_spai_build")

extern "C" pic_status pic_spai_get(const pic_mesh *pm, int32_t *free_edges, int64_t *indptr,
                                   int32_t *indices, double *values) try {
    if (!pm || !pm->h.have_spai) {
        set_error("pic_spai_get: no SPAI built");
        return PIC_ERR_STATE;
    }
    const HostMesh &m = pm->h;
    if (free_edges) std::copy(m.free_edges.begin(), m.free_edges.end(), free_edges);
    if (indptr) std::copy(m.M_ptr.begin(), m.M_ptr.end(), indptr);
    if (indices) std::copy(m.M_idx.begin(), m.M_idx.end(), indices);
    if (values) std::copy(m.M_val.begin(), m.M_val.end(), values);
    return PIC_OK;
}
PIC_CATCH("pic_spai_get")

extern "C" pic_status pic_spai_info(const pic_mesh *pm, int64_t *nnz, double *residual_rms,
                                    double *residual_max) try {
    if (!pm || !pm->h.have_spai) {
        set_error("pic_spai_info: no SPAI built");
        return PIC_ERR_STATE;
    }
    const HostMesh &m = pm->h;
    const int64_t nf = (int64_t)m.free_edges.size();
    // R = A_ff M - I row by row (A_ff: star_eps restricted to the free edges), with a dense
    // accumulator over the free edges
    std::vector<double> acc(nf, 0.0);
    std::vector<char> mark(nf, 0);
    std::vector<int32_t> touched;
    touched.reserve(256);
    double ss = 0.0, mx = 0.0;
    for (int64_t i = 0; i < nf; i++) {
        const int32_t ei = m.free_edges[i];
        touched.push_back((int32_t)i);   // the identity's entry
        mark[i] = 1;
        for (int64_t q = m.eps_ptr[ei]; q < m.eps_ptr[ei + 1]; q++) {
            const int32_t k = m.free_of_edge[m.eps_idx[q]];
            if (k < 0) continue;
            const double a = m.eps_val[q];
            for (int64_t r = m.M_ptr[k]; r < m.M_ptr[k + 1]; r++) {
                const int32_t j = m.M_idx[r];
                if (!mark[j]) {
                    mark[j] = 1;
                    touched.push_back(j);
                }
                acc[j] += a * m.M_val[r];
            }
        }
        for (int32_t j : touched) {
            const double v = acc[j] - (j == i ? 1.0 : 0.0);
            ss += v * v;
            mx = std::max(mx, std::fabs(v));
            acc[j] = 0.0;
            mark[j] = 0;
        }
        touched.clear();
    }
    if (nnz) *nnz = (int64_t)m.M_val.size();
    if (residual_rms) *residual_rms = nf > 0 ? std::sqrt(ss / (double)nf) : 0.0;
    if (residual_max) *residual_max = mx;
    return PIC_OK;
}
PIC_CATCH("pic_spai_info")
