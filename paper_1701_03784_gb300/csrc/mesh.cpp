// Mesh topology, geometry and Hodge operators of the meridian plane (host side).
//
// Sec. 3.1 / App. D: edges oriented from the lower to the higher node index, D_curl rows
// per face with entries +-1, D_div rows per node.  App. B: the rho-weighted Hodge
// matrix star_eps_ij = eps0 int rho W_i . W_j dz drho and the diagonal star_mu^-1.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <numeric>

#include "pic_internal.h"

namespace pic {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

// Radon's 7-point rule on a triangle, exact for polynomials of degree 5: barycentric
// points and weights (weights sum to 1; integral = area * sum w f).
struct Quad7 {
    double l[7][3];
    double w[7];
    Quad7() {
        const double s15 = std::sqrt(15.0);
        const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
        const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
        int q = 0;
        l[q][0] = l[q][1] = l[q][2] = 1.0 / 3.0;
        w[q++] = 9.0 / 40.0;
        const double as[2] = {a1, a2}, ws[2] = {w1, w2};
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) {
                for (int i = 0; i < 3; i++) l[q][i] = as[r];
                l[q][k] = 1.0 - 2.0 * as[r];
                w[q++] = ws[r];
            }
    }
};

// rho-weighted edge-element mass matrix of one triangle: the integrand
// rho (lambda_a grad lambda_b - lambda_b grad lambda_a) . (...) is cubic in lambda.
static void local_star_eps(const HostMesh &m, int64_t t, double eps0, double T[3][3]) {
    static const Quad7 Q;
    const int32_t *n3 = &m.tri[3 * t];
    const double *g = &m.grad[6 * t];
    double rho[3];
    for (int k = 0; k < 3; k++) rho[k] = m.zr[2 * n3[k] + 1];
    int ta[3], hb[3];
    for (int k = 0; k < 3; k++) edge_tail_head(n3, k, &ta[k], &hb[k]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[i][j] = 0.0;
    for (int q = 0; q < 7; q++) {
        const double *l = Q.l[q];
        double r = l[0] * rho[0] + l[1] * rho[1] + l[2] * rho[2];
        double W[3][2];
        for (int k = 0; k < 3; k++)
            for (int d = 0; d < 2; d++)
                W[k][d] = l[ta[k]] * g[2 * hb[k] + d] - l[hb[k]] * g[2 * ta[k] + d];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                T[i][j] += Q.w[q] * r * (W[i][0] * W[j][0] + W[i][1] * W[j][1]);
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[i][j] *= eps0 * m.area[t];
}

void build_locator(HostMesh &m) {
    double z0 = 1e300, z1 = -1e300, r0 = 1e300, r1 = -1e300, asum = 0;
    for (int64_t i = 0; i < m.N0; i++) {
        z0 = std::min(z0, m.zr[2 * i]);
        z1 = std::max(z1, m.zr[2 * i]);
        r0 = std::min(r0, m.zr[2 * i + 1]);
        r1 = std::max(r1, m.zr[2 * i + 1]);
    }
    for (int64_t t = 0; t < m.N2; t++) asum += m.area[t];
    double h = 2.0 * std::sqrt(asum / (double)m.N2);
    m.bb_z0 = z0;
    m.bb_r0 = r0;
    m.bb_h = h;
    m.bb_nz = std::max<int64_t>(1, (int64_t)std::ceil((z1 - z0) / h) + 1);
    m.bb_nr = std::max<int64_t>(1, (int64_t)std::ceil((r1 - r0) / h) + 1);
    std::vector<int64_t> cnt(m.bb_nz * m.bb_nr + 1, 0);
    auto cell_range = [&](int64_t t, int64_t &iz0, int64_t &iz1, int64_t &ir0, int64_t &ir1) {
        double a = 1e300, b = -1e300, c = 1e300, d = -1e300;
        for (int k = 0; k < 3; k++) {
            int32_t n = m.tri[3 * t + k];
            a = std::min(a, m.zr[2 * n]);
            b = std::max(b, m.zr[2 * n]);
            c = std::min(c, m.zr[2 * n + 1]);
            d = std::max(d, m.zr[2 * n + 1]);
        }
        iz0 = std::clamp<int64_t>((int64_t)std::floor((a - z0) / h), 0, m.bb_nz - 1);
        iz1 = std::clamp<int64_t>((int64_t)std::floor((b - z0) / h), 0, m.bb_nz - 1);
        ir0 = std::clamp<int64_t>((int64_t)std::floor((c - r0) / h), 0, m.bb_nr - 1);
        ir1 = std::clamp<int64_t>((int64_t)std::floor((d - r0) / h), 0, m.bb_nr - 1);
    };
    for (int64_t t = 0; t < m.N2; t++) {
        int64_t a, b, c, d;
        cell_range(t, a, b, c, d);
        for (int64_t iz = a; iz <= b; iz++)
            for (int64_t ir = c; ir <= d; ir++) cnt[iz * m.bb_nr + ir + 1]++;
    }
    for (size_t i = 1; i < cnt.size(); i++) cnt[i] += cnt[i - 1];
    m.bb_ptr = cnt;
    m.bb_tri.assign(cnt.back(), 0);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t t = 0; t < m.N2; t++) {
        int64_t a, b, c, d;
        cell_range(t, a, b, c, d);
        for (int64_t iz = a; iz <= b; iz++)
            for (int64_t ir = c; ir <= d; ir++) m.bb_tri[fill[iz * m.bb_nr + ir]++] = (int32_t)t;
    }
}

// barycentric coordinate k: signed area of (p, p_{k+1}, p_{k+2}) over the triangle's
static void bary(const HostMesh &m, int64_t t, double z, double r, double lam[3]) {
    const int32_t *n3 = &m.tri[3 * t];
    for (int k = 0; k < 3; k++) {
        const double *pa = &m.zr[2 * n3[(k + 1) % 3]];
        const double *pb = &m.zr[2 * n3[(k + 2) % 3]];
        lam[k] = ((pa[0] - z) * (pb[1] - r) - (pb[0] - z) * (pa[1] - r)) / (2.0 * m.area[t]);
    }
}

int32_t locate_point(const HostMesh &m, double z, double rho, double lam[3]) {
    int64_t iz = (int64_t)std::floor((z - m.bb_z0) / m.bb_h);
    int64_t ir = (int64_t)std::floor((rho - m.bb_r0) / m.bb_h);
    if (iz < 0 || ir < 0 || iz >= m.bb_nz || ir >= m.bb_nr) return -1;
    int64_t c = iz * m.bb_nr + ir;
    int32_t best = -1;
    double best_min = -1e300;
    for (int64_t k = m.bb_ptr[c]; k < m.bb_ptr[c + 1]; k++) {
        int32_t t = m.bb_tri[k];
        double l[3];
        bary(m, t, z, rho, l);
        double mn = std::min(l[0], std::min(l[1], l[2]));
        if (mn > best_min || (mn == best_min && t < best)) {
            best_min = mn;
            best = t;
        }
    }
    if (best < 0 || best_min < -1e-12) return -1;
    bary(m, best, z, rho, lam);
    return best;
}

}  // namespace pic

using namespace pic;

extern "C" const char *pic_last_error(void) { return pic::g_err.c_str(); }

extern "C" pic_status pic_mesh_create(const double *nodes_zr, int64_t n_nodes,
                                      const int32_t *tris, int64_t n_tris,
                                      const int32_t *bedge_nodes, const int32_t *bedge_tag,
                                      int64_t n_bedges, const pic_units *u, pic_mesh **out) try {
    if (!nodes_zr || !tris || !u || !out || n_nodes < 3 || n_tris < 1 || n_bedges < 0 ||
        (n_bedges > 0 && (!bedge_nodes || !bedge_tag))) {
        set_error("pic_mesh_create: null pointer or bad size");
        return PIC_ERR_ARG;
    }
    if (n_nodes >= (int64_t)1 << 31 || n_tris >= (int64_t)1 << 30) {
        set_error("pic_mesh_create: mesh too large for 32-bit indices");
        return PIC_ERR_ARG;
    }
    if (!(u->eps0 > 0) || !(u->mu0 > 0) || !(u->c > 0) ||
        (u->precision != PIC_FP64 && u->precision != PIC_FP32) || u->walk_cap < 0 ||
        u->walk_cap > PIC_WALK_CAP_MAX) {
        set_error("pic_mesh_create: bad units");
        return PIC_ERR_ARG;
    }
    pic_mesh *pm = new (std::nothrow) pic_mesh;
    if (!pm) {
        set_error("pic_mesh_create: out of host memory");
        return PIC_ERR_OOM;
    }
    HostMesh &m = pm->h;
    m.units = *u;
    if (m.units.walk_cap == 0) m.units.walk_cap = 16;
    m.N0 = n_nodes;
    m.N2 = n_tris;
    m.zr.assign(nodes_zr, nodes_zr + 2 * n_nodes);
    for (int64_t i = 0; i < n_nodes; i++)
        if (!(m.zr[2 * i + 1] >= 0.0) || !std::isfinite(m.zr[2 * i])) {
            set_error("pic_mesh_create: node %lld has rho < 0 or a non-finite coordinate",
                      (long long)i);
            delete pm;
            return PIC_ERR_ARG;
        }
    m.tri.assign(tris, tris + 3 * n_tris);
    m.area.resize(n_tris);
    m.grad.resize(6 * n_tris);
    for (int64_t t = 0; t < n_tris; t++) {
        int32_t *n3 = &m.tri[3 * t];
        for (int k = 0; k < 3; k++)
            if (n3[k] < 0 || n3[k] >= n_nodes) {
                set_error("pic_mesh_create: triangle %lld has a bad node index", (long long)t);
                delete pm;
                return PIC_ERR_ARG;
            }
        const double *p0 = &m.zr[2 * n3[0]], *p1 = &m.zr[2 * n3[1]], *p2 = &m.zr[2 * n3[2]];
        double s2 = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]);
        if (s2 == 0.0 || n3[0] == n3[1] || n3[1] == n3[2] || n3[0] == n3[2]) {
            set_error("pic_mesh_create: triangle %lld is degenerate", (long long)t);
            delete pm;
            return PIC_ERR_MESH;
        }
        if (s2 < 0) std::swap(n3[1], n3[2]);
        double A = 0.5 * std::fabs(s2);
        m.area[t] = A;
        for (int k = 0; k < 3; k++) {
            const double *pa = &m.zr[2 * n3[(k + 1) % 3]];
            const double *pb = &m.zr[2 * n3[(k + 2) % 3]];
            m.grad[6 * t + 2 * k + 0] = (pa[1] - pb[1]) / (2.0 * A);
            m.grad[6 * t + 2 * k + 1] = (pb[0] - pa[0]) / (2.0 * A);
        }
    }

    // edges: sort (lo, hi) keys of all local edges
    std::vector<std::pair<uint64_t, int64_t>> keys(3 * n_tris);
    for (int64_t t = 0; t < n_tris; t++)
        for (int k = 0; k < 3; k++) {
            uint64_t a = (uint64_t)m.tri[3 * t + (k + 1) % 3];
            uint64_t b = (uint64_t)m.tri[3 * t + (k + 2) % 3];
            uint64_t lo = std::min(a, b), hi = std::max(a, b);
            keys[3 * t + k] = {lo * (uint64_t)n_nodes + hi, 3 * t + k};
        }
    std::sort(keys.begin(), keys.end());
    m.tri_edge.assign(3 * n_tris, -1);
    m.tri_nbr.assign(3 * n_tris, -1);
    std::vector<int64_t> ecount;
    for (size_t i = 0; i < keys.size();) {
        size_t j = i;
        while (j < keys.size() && keys[j].first == keys[i].first) j++;
        int64_t e = (int64_t)m.edge_nodes.size() / 2;
        if (j - i > 2) {
            set_error("pic_mesh_create: an edge is shared by more than two triangles");
            delete pm;
            return PIC_ERR_MESH;
        }
        m.edge_nodes.push_back((int32_t)(keys[i].first / (uint64_t)n_nodes));
        m.edge_nodes.push_back((int32_t)(keys[i].first % (uint64_t)n_nodes));
        m.edge_face.push_back(-1);
        m.edge_face.push_back(-1);
        m.edge_face_sign.push_back(0);
        m.edge_face_sign.push_back(0);
        for (size_t q = i; q < j; q++) {
            int64_t t = keys[q].second / 3;
            int k = (int)(keys[q].second % 3);
            m.tri_edge[3 * t + k] = (int32_t)e;
            int32_t a = m.tri[3 * t + (k + 1) % 3], b = m.tri[3 * t + (k + 2) % 3];
            m.edge_face[2 * e + (q - i)] = (int32_t)t;
            m.edge_face_sign[2 * e + (q - i)] = (int8_t)(a < b ? 1 : -1);
        }
        if (j - i == 2) {
            int64_t t0 = keys[i].second / 3, t1 = keys[i + 1].second / 3;
            // both triangles are counter-clockwise: a conforming pair runs the shared edge in
            // opposite directions; the same direction means they overlap
            if (m.edge_face_sign[2 * e] == m.edge_face_sign[2 * e + 1]) {
                set_error("pic_mesh_create: triangles %lld and %lld overlap at a shared edge",
                          (long long)t0, (long long)t1);
                delete pm;
                return PIC_ERR_MESH;
            }
            m.tri_nbr[keys[i].second] = (int32_t)t1;
            m.tri_nbr[keys[i + 1].second] = (int32_t)t0;
        }
        ecount.push_back((int64_t)(j - i));
        i = j;
    }
    m.N1 = (int64_t)ecount.size();

    // boundary tags
    m.edge_tag.assign(m.N1, 0);
    for (int64_t b = 0; b < n_bedges; b++) {
        int32_t a = bedge_nodes[2 * b], c = bedge_nodes[2 * b + 1];
        int32_t tag = bedge_tag[b];
        if (a < 0 || c < 0 || a >= n_nodes || c >= n_nodes || a == c ||
            (tag != PIC_BC_PEC && tag != PIC_BC_AXIS && tag != PIC_BC_ABSORB)) {
            set_error("pic_mesh_create: bad boundary edge %lld", (long long)b);
            delete pm;
            return PIC_ERR_ARG;
        }
        uint64_t key = (uint64_t)std::min(a, c) * (uint64_t)n_nodes + (uint64_t)std::max(a, c);
        auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(key, (int64_t)-1));
        if (it == keys.end() || it->first != key) {
            set_error("pic_mesh_create: boundary edge %lld is not a mesh edge", (long long)b);
            delete pm;
            return PIC_ERR_MESH;
        }
        int64_t e = m.tri_edge[it->second];
        if (ecount[e] != 1 || m.edge_tag[e] != 0) {
            set_error("pic_mesh_create: boundary edge %lld is interior or listed twice",
                      (long long)b);
            delete pm;
            return PIC_ERR_MESH;
        }
        m.edge_tag[e] = tag;
    }
    for (int64_t e = 0; e < m.N1; e++)
        if (ecount[e] == 1 && m.edge_tag[e] == 0) {
            set_error("pic_mesh_create: mesh boundary edge %lld (%d,%d) has no tag",
                      (long long)e, m.edge_nodes[2 * e], m.edge_nodes[2 * e + 1]);
            delete pm;
            return PIC_ERR_MESH;
        }
    m.free_of_edge.assign(m.N1, -1);
    m.node_on_pec.assign(m.N0, 0);
    for (int64_t e = 0; e < m.N1; e++) {
        if (m.edge_tag[e] == PIC_BC_PEC) {
            m.node_on_pec[m.edge_nodes[2 * e]] = 1;
            m.node_on_pec[m.edge_nodes[2 * e + 1]] = 1;
        } else {
            m.free_of_edge[e] = (int32_t)m.free_edges.size();
            m.free_edges.push_back((int32_t)e);
        }
    }

    // star_mu^-1: (1/mu0) int rho W2 W2 = rho_bar / (mu0 A)
    m.mu_inv.resize(n_tris);
    for (int64_t t = 0; t < n_tris; t++) {
        double rb = 0;
        for (int k = 0; k < 3; k++) rb += m.zr[2 * m.tri[3 * t + k] + 1];
        m.mu_inv[t] = (rb / 3.0) / (u->mu0 * m.area[t]);
    }

    // star_eps assembly: triplets sorted by (row, col) and merged
    std::vector<std::pair<uint64_t, double>> trip;
    trip.reserve(9 * n_tris);
    for (int64_t t = 0; t < n_tris; t++) {
        double T[3][3];
        local_star_eps(m, t, u->eps0, T);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                trip.push_back({(uint64_t)m.tri_edge[3 * t + i] * (uint64_t)m.N1 +
                                    (uint64_t)m.tri_edge[3 * t + j],
                                T[i][j]});
    }
    std::sort(trip.begin(), trip.end(),
              [](const auto &x, const auto &y) { return x.first < y.first; });
    m.eps_ptr.assign(m.N1 + 1, 0);
    for (size_t i = 0; i < trip.size();) {
        size_t j = i;
        double v = 0;
        while (j < trip.size() && trip[j].first == trip[i].first) v += trip[j++].second;
        int64_t row = (int64_t)(trip[i].first / (uint64_t)m.N1);
        m.eps_idx.push_back((int32_t)(trip[i].first % (uint64_t)m.N1));
        m.eps_val.push_back(v);
        m.eps_ptr[row + 1]++;
        i = j;
    }
    for (int64_t r = 0; r < m.N1; r++) m.eps_ptr[r + 1] += m.eps_ptr[r];

    build_locator(m);
    *out = pm;
    return PIC_OK;
}
PIC_CATCH("pic_mesh_create")

extern "C" pic_status pic_mesh_info(const pic_mesh *m, int64_t *n_nodes, int64_t *n_edges,
                                    int64_t *n_tris, int64_t *n_free_edges,
                                    int64_t *spai_nnz) try {
    if (!m) {
        set_error("pic_mesh_info: null mesh");
        return PIC_ERR_ARG;
    }
    if (n_nodes) *n_nodes = m->h.N0;
    if (n_edges) *n_edges = m->h.N1;
    if (n_tris) *n_tris = m->h.N2;
    if (n_free_edges) *n_free_edges = (int64_t)m->h.free_edges.size();
    if (spai_nnz) *spai_nnz = m->h.have_spai ? (int64_t)m->h.M_val.size() : 0;
    return PIC_OK;
}
PIC_CATCH("pic_mesh_info")

extern "C" pic_status pic_mesh_edges(const pic_mesh *m, int32_t *edge_nodes) try {
    if (!m || !edge_nodes) {
        set_error("pic_mesh_edges: null pointer");
        return PIC_ERR_ARG;
    }
    std::copy(m->h.edge_nodes.begin(), m->h.edge_nodes.end(), edge_nodes);
    return PIC_OK;
}
PIC_CATCH("pic_mesh_edges")

extern "C" void pic_mesh_destroy(pic_mesh *m) { delete m; }
