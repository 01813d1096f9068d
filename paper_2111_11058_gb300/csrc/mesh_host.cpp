// mesh_host.cpp -- RWG edge table and cell division (paper Sec. II-B, RWG
// functions; Sec. III-A, cells: every edge in exactly one cell).
//
// Canonical edges: unique vertex pairs (u < v) in lexicographic order; the
// plus triangle is the one whose counter-clockwise order runs u -> v.  Local
// edge a of a triangle joins its vertices (a+1)%3 and (a+2)%3 (free vertex a).
// Internal order: edges sorted by (cell, canonical index).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>

#include "internal.cuh"

namespace cbfm {

namespace {

uint64_t key(int32_t u, int32_t v) { return (uint64_t(uint32_t(u)) << 32) | uint32_t(v); }

void rcb(const std::vector<double> &mid, std::vector<int64_t> ids, int first, int mcount,
         std::vector<int32_t> &cell) {
    if (mcount == 1) {
        for (int64_t e : ids) cell[e] = first;
        return;
    }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t e : ids)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], mid[3 * e + d]);
            hi[d] = std::max(hi[d], mid[3 * e + d]);
        }
    int ax = 0;
    double best = hi[0] - lo[0];
    for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > best) { best = hi[d] - lo[d]; ax = d; }
    std::sort(ids.begin(), ids.end(), [&](int64_t a, int64_t b) {
        double ca = mid[3 * a + ax], cb = mid[3 * b + ax];
        if (ca != cb) return ca < cb;
        return a < b;
    });
    int ml = mcount / 2;
    int64_t nl = (int64_t)std::floor((double)ids.size() * ml / mcount + 0.5);
    std::vector<int64_t> left(ids.begin(), ids.begin() + nl), right(ids.begin() + nl, ids.end());
    rcb(mid, left, first, ml, cell);
    rcb(mid, right, first + ml, mcount - ml, cell);
}

}  // namespace

void build_host_mesh(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                     const int32_t *edge_cell, int32_t ncell, int32_t partition, HostMesh &hm) {
    CBFM_REQUIRE(nv >= 4 && nt >= 4, "mesh needs at least 4 vertices and 4 triangles");
    CBFM_REQUIRE(nt < (int64_t(1) << 30) && nv < (int64_t(1) << 30), "mesh too large for int32 indices");
    CBFM_REQUIRE(ncell >= 1, "ncell must be >= 1");
    hm.nv = nv;
    hm.nt = nt;
    hm.verts.assign(verts, verts + 3 * nv);
    hm.tris.assign(tris, tris + 3 * nt);
    for (int64_t i = 0; i < 3 * nt; ++i) CBFM_REQUIRE(tris[i] >= 0 && tris[i] < nv, "triangle vertex index out of range");

    // directed edges -> (triangle, local index)
    std::unordered_map<uint64_t, int64_t> directed;
    directed.reserve(size_t(3 * nt) * 2);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            int32_t u = tris[3 * t + (a + 1) % 3], v = tris[3 * t + (a + 2) % 3];
            CBFM_REQUIRE(u != v, "degenerate triangle");
            auto ins = directed.emplace(key(u, v), 3 * t + a);
            CBFM_REQUIRE(ins.second, "non-manifold or inconsistently oriented mesh");
        }
    std::vector<uint64_t> und;
    und.reserve(directed.size() / 2 + 1);
    for (auto &kv : directed) {
        int32_t u = int32_t(kv.first >> 32), v = int32_t(kv.first & 0xffffffffu);
        CBFM_REQUIRE(directed.count(key(v, u)), "open mesh: edge with a single triangle");
        if (u < v) und.push_back(kv.first);
    }
    std::sort(und.begin(), und.end());
    int64_t ne = (int64_t)und.size();
    CBFM_REQUIRE(ne * 2 == 3 * nt, "mesh is not a closed 2-manifold");
    hm.ne = ne;
    hm.canon_u.resize(ne);
    hm.canon_v.resize(ne);
    for (int64_t e = 0; e < ne; ++e) {
        hm.canon_u[e] = int32_t(und[e] >> 32);
        hm.canon_v[e] = int32_t(und[e] & 0xffffffffu);
    }

    // cells
    hm.cell_of_canon.assign(ne, 0);
    if (edge_cell) {
        for (int64_t e = 0; e < ne; ++e) {
            CBFM_REQUIRE(edge_cell[e] >= 0 && edge_cell[e] < ncell, "edge_cell out of range");
            hm.cell_of_canon[e] = edge_cell[e];
        }
    } else {
        std::vector<double> mid(3 * ne);
        for (int64_t e = 0; e < ne; ++e)
            for (int d = 0; d < 3; ++d)
                mid[3 * e + d] = 0.5 * (verts[3 * hm.canon_u[e] + d] + verts[3 * hm.canon_v[e] + d]);
        if (partition == 0) {
            CBFM_REQUIRE(ncell == 8, "octant partition needs ncell == 8");
            double ext = 0;
            for (int64_t i = 0; i < 3 * nv; ++i) ext = std::max(ext, std::fabs(verts[i]));
            double thr = -1e-12 * ext;
            for (int64_t e = 0; e < ne; ++e) {
                int c = 0;
                if (mid[3 * e + 0] < thr) c += 1;
                if (mid[3 * e + 1] < thr) c += 2;
                if (mid[3 * e + 2] < thr) c += 4;
                hm.cell_of_canon[e] = c;
            }
        } else {
            CBFM_REQUIRE(ncell <= ne, "more cells than edges");
            std::vector<int64_t> ids(ne);
            std::iota(ids.begin(), ids.end(), 0);
            rcb(mid, ids, 0, ncell, hm.cell_of_canon);
        }
    }
    hm.ncell = ncell;

    // internal order: (cell, canonical)
    std::vector<int32_t> order(ne);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return hm.cell_of_canon[a] < hm.cell_of_canon[b]; });
    hm.canon_of_int = order;
    hm.int_of_canon.assign(ne, 0);
    for (int64_t i = 0; i < ne; ++i) hm.int_of_canon[order[i]] = int32_t(i);
    hm.cell_off.assign(ncell + 1, 0);
    for (int64_t e = 0; e < ne; ++e) hm.cell_off[hm.cell_of_canon[e] + 1]++;
    for (int c = 0; c < ncell; ++c) {
        CBFM_REQUIRE(hm.cell_off[c + 1] > 0, "empty cell " + std::to_string(c));
        hm.cell_off[c + 1] += hm.cell_off[c];
    }

    // RWG tables in internal order
    hm.edge_tri.assign(2 * ne, 0);
    hm.edge_loc.assign(2 * ne, 0);
    hm.edge_len.assign(ne, 0.0);
    hm.tri_edge.assign(3 * nt, -1);
    hm.tri_sign.assign(3 * nt, 0);
    for (int64_t ce = 0; ce < ne; ++ce) {
        int32_t ie = hm.int_of_canon[ce];
        int32_t u = hm.canon_u[ce], v = hm.canon_v[ce];
        int64_t tp = directed[key(u, v)], tm = directed[key(v, u)];
        hm.edge_tri[2 * ie] = int32_t(tp / 3);
        hm.edge_loc[2 * ie] = int32_t(tp % 3);
        hm.edge_tri[2 * ie + 1] = int32_t(tm / 3);
        hm.edge_loc[2 * ie + 1] = int32_t(tm % 3);
        hm.tri_edge[tp] = ie;
        hm.tri_sign[tp] = 1;
        hm.tri_edge[tm] = ie;
        hm.tri_sign[tm] = -1;
        double dx = verts[3 * v] - verts[3 * u], dy = verts[3 * v + 1] - verts[3 * u + 1],
               dz = verts[3 * v + 2] - verts[3 * u + 2];
        hm.edge_len[ie] = std::sqrt(dx * dx + dy * dy + dz * dz);
    }
}

}  // namespace cbfm
