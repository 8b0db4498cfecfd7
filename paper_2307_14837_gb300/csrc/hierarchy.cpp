// Host construction of level L+1 and the DNN-MG patch data (Sec. 5.2).
//
// A patch is one coarse cell with the 27 nodes of its uniform refinement;
// dof(P, iota) of Sec. 5.2 is patch_map[P][iota] with iota = a + 3b + 9c.
// Fine nodes: coarse vertices keep their numbers, then one node per coarse
// edge, face and cell, numbered by first appearance (cells in order, local
// edges / faces in the order of kEdges / kFaces).  The valence of a node is
// the number of patches that contain it (mu = 1 / valence in Eq. (15)).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "internal.h"

namespace dnnmg {
namespace {

// local edges: xi-edges, eta-edges, zeta-edges
const int kEdges[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                           {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
// local faces xi=0, xi=1, eta=0, eta=1, zeta=0, zeta=1; vertices listed
// lexicographically in the face's two free coordinates
const int kFaces[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5},
                          {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};

struct FaceKey {
    uint64_t lo, hi;
    bool operator==(const FaceKey& o) const { return lo == o.lo && hi == o.hi; }
};
struct FaceHash {
    size_t operator()(const FaceKey& k) const {
        uint64_t x = k.lo * 0x9E3779B97F4A7C15ull ^ (k.hi + 0x632BE59BD9B4E019ull + (k.lo << 6));
        x ^= x >> 31;
        return static_cast<size_t>(x * 0xBF58476D1CE4E5B9ull);
    }
};
struct EdgeHash {
    size_t operator()(uint64_t k) const {
        k ^= k >> 33;
        k *= 0xFF51AFD7ED558CCDull;
        k ^= k >> 33;
        return static_cast<size_t>(k);
    }
};

FaceKey face_key(const int32_t* cv, int f) {
    std::array<uint32_t, 4> v;
    for (int i = 0; i < 4; ++i) v[i] = static_cast<uint32_t>(cv[kFaces[f][i]]);
    std::sort(v.begin(), v.end());
    return FaceKey{(uint64_t(v[0]) << 32) | v[1], (uint64_t(v[2]) << 32) | v[3]};
}

uint64_t edge_key(int32_t a, int32_t b) {
    if (a > b) std::swap(a, b);
    return (uint64_t(uint32_t(a)) << 32) | uint32_t(b);
}

// priority of boundary kinds: outflow (3) < wall (1) < driven (2)
int prio(int kind) { return kind == 3 ? 0 : kind == 1 ? 1 : kind == 2 ? 2 : -1; }
int kind_of_prio(int p) { return p == 0 ? 3 : p == 1 ? 1 : 2; }

// What patch node iota refines: 0 vertex, 1 edge, 2 face, 3 cell; and which one.
struct LocalEntity {
    int type, index;
};
LocalEntity local_entity(int iota) {
    const int a = iota % 3, b = (iota / 3) % 3, c = iota / 9;
    const int mids = (a == 1) + (b == 1) + (c == 1);
    if (mids == 0) return {0, a / 2 + 2 * (b / 2) + 4 * (c / 2)};
    if (mids == 1) {
        if (a == 1) return {1, b / 2 + 2 * (c / 2)};
        if (b == 1) return {1, 4 + a / 2 + 2 * (c / 2)};
        return {1, 8 + a / 2 + 2 * (b / 2)};
    }
    if (mids == 2) {
        if (a != 1) return {2, a / 2};
        if (b != 1) return {2, 2 + b / 2};
        return {2, 4 + c / 2};
    }
    return {3, 0};
}

}  // namespace

namespace {

// Level L+1 of a mesh and its 27-node patches (J = 1).
dnnmg_status build_one(const dnnmg_mesh_desc* mesh, int n_geo, HostHierarchy* h, std::string* err) {
    if (!mesh || !mesh->xyz || !mesh->cell_vertices || !mesh->vertex_bc || mesh->n_vertices <= 0 ||
        mesh->n_cells <= 0) {
        *err = "mesh: null array or non-positive size";
        return DNNMG_EINVAL;
    }
    const int64_t nv = mesh->n_vertices, nc = mesh->n_cells;
    // 27 nc node references must fit int32 CSR entries
    if (nc > (int64_t(1) << 31) / 32) {
        *err = "mesh: too many cells";
        return DNNMG_EINVAL;
    }
    h->nv = nv;
    h->nc = nc;
    h->J = 1;
    h->npn = 27;
    h->xyz_c.assign(mesh->xyz, mesh->xyz + 3 * nv);
    h->cells.assign(mesh->cell_vertices, mesh->cell_vertices + 8 * nc);
    h->bc_c.assign(mesh->vertex_bc, mesh->vertex_bc + nv);
    for (int64_t v = 0; v < nv; ++v) {
        if (h->bc_c[v] < 0 || h->bc_c[v] > 3) {
            *err = "mesh: vertex_bc outside 0..3";
            return DNNMG_EINVAL;
        }
    }
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t* cv = &h->cells[8 * c];
        for (int k = 0; k < 8; ++k) {
            if (cv[k] < 0 || cv[k] >= nv) {
                *err = "mesh: cell vertex index out of range";
                return DNNMG_EINVAL;
            }
            for (int l = 0; l < k; ++l)
                if (cv[l] == cv[k]) {
                    *err = "mesh: cell with a repeated vertex";
                    return DNNMG_EINVAL;
                }
        }
    }

    // ---- boundary faces and their kinds
    std::unordered_map<FaceKey, int32_t, FaceHash> face_count;
    face_count.reserve(size_t(4 * nc));
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < 6; ++f) face_count[face_key(&h->cells[8 * c], f)]++;
    std::unordered_map<FaceKey, int32_t, FaceHash> bface_kind;
    for (const auto& kv : face_count) {
        if (kv.second != 1) continue;
        const uint32_t v[4] = {uint32_t(kv.first.lo >> 32), uint32_t(kv.first.lo),
                               uint32_t(kv.first.hi >> 32), uint32_t(kv.first.hi)};
        int p = 3;
        for (int i = 0; i < 4; ++i) {
            const int k = h->bc_c[v[i]];
            if (k == 0) {
                *err = "mesh: boundary face with an interior-marked vertex";
                return DNNMG_EINVAL;
            }
            p = std::min(p, prio(k));
        }
        bface_kind[kv.first] = kind_of_prio(p);
    }
    std::unordered_map<uint64_t, int32_t, EdgeHash> bedge_prio;
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t* cv = &h->cells[8 * c];
        for (int f = 0; f < 6; ++f) {
            auto it = bface_kind.find(face_key(cv, f));
            if (it == bface_kind.end()) continue;
            const int p = prio(it->second);
            const int32_t* fv = kFaces[f];
            const int pairs[4][2] = {{0, 1}, {2, 3}, {0, 2}, {1, 3}};
            for (auto& pr : pairs) {
                const uint64_t k = edge_key(cv[fv[pr[0]]], cv[fv[pr[1]]]);
                auto e = bedge_prio.find(k);
                if (e == bedge_prio.end())
                    bedge_prio[k] = p;
                else
                    e->second = std::max(e->second, p);
            }
        }
    }

    // ---- number edges and faces by first appearance
    std::unordered_map<uint64_t, int32_t, EdgeHash> edge_id;
    edge_id.reserve(size_t(4 * nc));
    std::vector<std::array<int32_t, 2>> edge_par;
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t* cv = &h->cells[8 * c];
        for (int e = 0; e < 12; ++e) {
            const int32_t a = cv[kEdges[e][0]], b = cv[kEdges[e][1]];
            auto ins = edge_id.emplace(edge_key(a, b), int32_t(nv + edge_par.size()));
            if (ins.second) edge_par.push_back({a, b});
        }
    }
    const int64_t ne = int64_t(edge_par.size());
    std::unordered_map<FaceKey, int32_t, FaceHash> face_id;
    face_id.reserve(size_t(4 * nc));
    std::vector<std::array<int32_t, 4>> face_par;
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t* cv = &h->cells[8 * c];
        for (int f = 0; f < 6; ++f) {
            auto ins = face_id.emplace(face_key(cv, f), int32_t(nv + ne + face_par.size()));
            if (ins.second)
                face_par.push_back({cv[kFaces[f][0]], cv[kFaces[f][1]], cv[kFaces[f][2]], cv[kFaces[f][3]]});
        }
    }
    const int64_t nf = int64_t(face_par.size());
    const int64_t n_fine = nv + ne + nf + nc;
    if (n_fine >= (int64_t(1) << 31)) {
        *err = "mesh: too many fine nodes for int32 indices";
        return DNNMG_EINVAL;
    }
    h->ne = ne;
    h->nf = nf;
    h->n_fine = n_fine;

    // ---- patch map
    h->patch_map.resize(size_t(27 * nc));
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t* cv = &h->cells[8 * c];
        for (int iota = 0; iota < 27; ++iota) {
            const LocalEntity le = local_entity(iota);
            int32_t id;
            if (le.type == 0)
                id = cv[le.index];
            else if (le.type == 1)
                id = edge_id.at(edge_key(cv[kEdges[le.index][0]], cv[kEdges[le.index][1]]));
            else if (le.type == 2)
                id = face_id.at(face_key(cv, le.index));
            else
                id = int32_t(nv + ne + nf + c);
            h->patch_map[size_t(27 * c + iota)] = id;
        }
    }

    // ---- kinds, coordinates
    h->kind_f.assign(size_t(n_fine), 0);
    h->xyz_f.assign(size_t(3 * n_fine), 0.0);
    for (int64_t v = 0; v < nv; ++v) {
        h->kind_f[v] = h->bc_c[v];
        for (int d = 0; d < 3; ++d) h->xyz_f[3 * v + d] = h->xyz_c[3 * v + d];
    }
    for (int64_t i = 0; i < ne; ++i) {
        const auto& e = edge_par[i];
        auto it = bedge_prio.find(edge_key(e[0], e[1]));
        h->kind_f[nv + i] = it == bedge_prio.end() ? 0 : kind_of_prio(it->second);
        for (int d = 0; d < 3; ++d)
            h->xyz_f[3 * (nv + i) + d] = (h->xyz_c[3 * e[0] + d] + h->xyz_c[3 * e[1] + d]) / 2.0;
    }
    for (int64_t i = 0; i < nf; ++i) {
        const auto& f = face_par[i];
        FaceKey key;
        {
            std::array<uint32_t, 4> v = {uint32_t(f[0]), uint32_t(f[1]), uint32_t(f[2]), uint32_t(f[3])};
            std::sort(v.begin(), v.end());
            key = FaceKey{(uint64_t(v[0]) << 32) | v[1], (uint64_t(v[2]) << 32) | v[3]};
        }
        auto it = bface_kind.find(key);
        h->kind_f[nv + ne + i] = it == bface_kind.end() ? 0 : it->second;
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += h->xyz_c[3 * f[k] + d];
            h->xyz_f[3 * (nv + ne + i) + d] = s / 4.0;
        }
    }
    for (int64_t c = 0; c < nc; ++c) {
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += h->xyz_c[3 * h->cells[8 * c + k] + d];
            h->xyz_f[3 * (nv + ne + nf + c) + d] = s / 8.0;
        }
    }

    // ---- valences and the node -> (patch, iota) CSR in patch order
    h->valence.assign(size_t(n_fine), 0);
    for (int64_t e = 0; e < 27 * nc; ++e) h->valence[h->patch_map[e]]++;
    h->node_ptr.assign(size_t(n_fine + 1), 0);
    for (int64_t j = 0; j < n_fine; ++j) h->node_ptr[j + 1] = h->node_ptr[j] + h->valence[j];
    h->node_idx.assign(size_t(27 * nc), 0);
    {
        std::vector<int32_t> fill(h->node_ptr.begin(), h->node_ptr.end() - 1);
        for (int64_t e = 0; e < 27 * nc; ++e) h->node_idx[fill[h->patch_map[e]]++] = int32_t(e);
    }
    // coarse vertex -> (patch, local vertex) CSR in patch order
    h->vert_ptr.assign(size_t(nv + 1), 0);
    for (int64_t e = 0; e < 8 * nc; ++e) h->vert_ptr[h->cells[e] + 1]++;
    for (int64_t v = 0; v < nv; ++v) h->vert_ptr[v + 1] += h->vert_ptr[v];
    h->vert_idx.assign(size_t(8 * nc), 0);
    {
        std::vector<int32_t> fill(h->vert_ptr.begin(), h->vert_ptr.end() - 1);
        for (int64_t e = 0; e < 8 * nc; ++e) h->vert_idx[fill[h->cells[e]]++] = int32_t(e);
    }

    // ---- geometry features of each coarse cell (Sec. 5.2, network inputs):
    // the 12 edge lengths; with n_geo = 24 also the 4 lengths of the space
    // diagonals (vertex k to vertex 7 - k, k = 0..3) and, for each vertex k,
    // the mean of the 3 interior angles between the faces that meet there
    // (radians; the angle between two faces along their common edge e is
    // the angle between the other two edges at k projected orthogonally to e)
    h->n_geo = n_geo;
    h->geo.assign(size_t(n_geo) * size_t(nc), 0.0);
    auto vec = [&](int32_t a, int32_t b, double* t) {
        for (int d = 0; d < 3; ++d) t[d] = h->xyz_c[3 * size_t(b) + d] - h->xyz_c[3 * size_t(a) + d];
    };
    auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t* cv = &h->cells[8 * c];
        double* g = &h->geo[size_t(n_geo) * size_t(c)];
        double t[3];
        for (int e = 0; e < 12; ++e) {
            vec(cv[kEdges[e][0]], cv[kEdges[e][1]], t);
            g[e] = std::sqrt(dot(t, t));
        }
        if (n_geo < 24) continue;
        for (int k = 0; k < 4; ++k) {
            vec(cv[k], cv[7 - k], t);
            g[12 + k] = std::sqrt(dot(t, t));
        }
        for (int k = 0; k < 8; ++k) {
            double ed[3][3];   // edges from vertex k along the three axes
            for (int a = 0; a < 3; ++a) vec(cv[k], cv[k ^ (1 << a)], ed[a]);
            double sum = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double* e = ed[a];
                const double* u = ed[(a + 1) % 3];
                const double* w = ed[(a + 2) % 3];
                const double ee = dot(e, e), ue = dot(u, e) / ee, we = dot(w, e) / ee;
                double up[3], wp[3];
                for (int d = 0; d < 3; ++d) {
                    up[d] = u[d] - ue * e[d];
                    wp[d] = w[d] - we * e[d];
                }
                double cs = dot(up, wp) / std::sqrt(dot(up, up) * dot(wp, wp));
                cs = cs > 1.0 ? 1.0 : (cs < -1.0 ? -1.0 : cs);
                sum += std::acos(cs);
            }
            g[16 + k] = sum / 3.0;
        }
    }
    return DNNMG_OK;
}

}  // namespace

dnnmg_status build_hierarchy(const dnnmg_mesh_desc* mesh, int n_geo, int J, HostHierarchy* h, std::string* err) {
    if (J == 1) return build_one(mesh, n_geo, h, err);
    if (J != 2) {
        *err = "patch levels must be 1 or 2";
        return DNNMG_EINVAL;
    }
    // J = 2: level L+2 is level L+1 refined by the same rules, with level
    // L+1 as a mesh whose cell 8 P + (ci + 2 cj + 4 ck) is child (ci, cj, ck)
    // of coarse cell P (vertices in lexicographic order)
    HostHierarchy h1;
    dnnmg_status st = build_one(mesh, n_geo, &h1, err);
    if (st != DNNMG_OK) return st;
    const int64_t nc = h1.nc;
    std::vector<int32_t> cells1(size_t(64 * nc));
    for (int64_t P = 0; P < nc; ++P)
        for (int child = 0; child < 8; ++child) {
            const int ci = child & 1, cj = (child >> 1) & 1, ck = (child >> 2) & 1;
            for (int k = 0; k < 8; ++k) {
                const int iota = (ci + (k & 1)) + 3 * (cj + ((k >> 1) & 1)) + 9 * (ck + ((k >> 2) & 1));
                cells1[size_t(8 * (8 * P + child) + k)] = h1.patch_map[size_t(27 * P + iota)];
            }
        }
    dnnmg_mesh_desc m1;
    m1.n_vertices = int32_t(h1.n_fine);
    m1.xyz = h1.xyz_f.data();
    m1.n_cells = int32_t(8 * nc);
    m1.cell_vertices = cells1.data();
    m1.vertex_bc = h1.kind_f.data();
    HostHierarchy h2;
    if ((st = build_one(&m1, 12, &h2, err)) != DNNMG_OK) return st;
    // the patch of coarse cell P: node (a, b, c) in {0..4}^3 is node
    // (a - 2 ci, b - 2 cj, c - 2 ck) of child (ci, cj, ck), ci = min(a / 2, 1)
    std::vector<int32_t> pm_mid = h1.patch_map, kind_mid = h1.kind_f, mid_ptr = h1.node_ptr, mid_idx = h1.node_idx;
    std::vector<double> xyz_mid = h1.xyz_f;
    const int64_t n_mid = h1.n_fine;
    *h = std::move(h1);
    h->n_mid = n_mid;
    h->patch_map_mid = std::move(pm_mid);
    h->kind_mid = std::move(kind_mid);
    h->xyz_mid = std::move(xyz_mid);
    h->mid_ptr = std::move(mid_ptr);
    h->mid_idx = std::move(mid_idx);
    h->J = 2;
    h->npn = 125;
    h->n_fine = h2.n_fine;
    h->kind_f = std::move(h2.kind_f);
    h->xyz_f = std::move(h2.xyz_f);
    h->patch_map.assign(size_t(125 * nc), 0);
    for (int64_t P = 0; P < nc; ++P)
        for (int iota = 0; iota < 125; ++iota) {
            const int a = iota % 5, b = (iota / 5) % 5, c = iota / 25;
            const int ci = std::min(a / 2, 1), cj = std::min(b / 2, 1), ck = std::min(c / 2, 1);
            const int child = ci + 2 * cj + 4 * ck;
            const int l = (a - 2 * ci) + 3 * (b - 2 * cj) + 9 * (c - 2 * ck);
            h->patch_map[size_t(125 * P + iota)] = h2.patch_map[size_t(27 * (8 * P + child) + l)];
        }
    // valences and the node -> (patch, iota) CSR in patch order
    const int64_t n_fine = h->n_fine;
    h->valence.assign(size_t(n_fine), 0);
    for (int64_t e = 0; e < 125 * nc; ++e) h->valence[h->patch_map[e]]++;
    h->node_ptr.assign(size_t(n_fine + 1), 0);
    for (int64_t j = 0; j < n_fine; ++j) h->node_ptr[j + 1] = h->node_ptr[j] + h->valence[j];
    h->node_idx.assign(size_t(125 * nc), 0);
    {
        std::vector<int32_t> fill(h->node_ptr.begin(), h->node_ptr.end() - 1);
        for (int64_t e = 0; e < 125 * nc; ++e) h->node_idx[fill[h->patch_map[e]]++] = int32_t(e);
    }
    return DNNMG_OK;
}

}  // namespace dnnmg

namespace dnnmg {

namespace {

// Cells in consecutive groups of 8 children (i + 2j + 4k) of a parent?  On
// success g27 holds the 27 nodes of each group (iota = a + 3b + 9c).
bool group_cells(const std::vector<int32_t>& cells, int64_t nc, std::vector<int32_t>* g27) {
    if (nc % 8 != 0 || nc == 0) return false;
    const int64_t ng = nc / 8;
    g27->assign(size_t(27 * ng), -1);
    for (int64_t g = 0; g < ng; ++g)
        for (int t = 0; t < 8; ++t)
            for (int k = 0; k < 8; ++k) {
                const int a = (t & 1) + (k & 1), b = ((t >> 1) & 1) + ((k >> 1) & 1),
                          c = ((t >> 2) & 1) + ((k >> 2) & 1);
                int32_t& slot = (*g27)[size_t(27 * g + a + 3 * b + 9 * c)];
                const int32_t v = cells[size_t(8 * (8 * g + t) + k)];
                if (slot < 0)
                    slot = v;
                else if (slot != v)
                    return false;
            }
    return true;
}

// Pinned pressure node, node CSR, block sparsity and block maps of a level
// whose groups, nodes and Dirichlet flags are set.
void finish_level(HostLevel* lv) {
    const int npg = lv->npg;
    const int64_t n = lv->n, ng = lv->ng;
    lv->pin = -1;
    if (lv->mean_zero_pressure)
        for (int64_t j = 0; j < n; ++j)
            if (!lv->dir[j]) {
                lv->pin = int32_t(j);
                break;
            }
    // node -> (group, local) in group order
    lv->node_ptr.assign(size_t(n + 1), 0);
    for (int64_t e = 0; e < ng * npg; ++e) lv->node_ptr[lv->groups[e] + 1]++;
    for (int64_t j = 0; j < n; ++j) lv->node_ptr[j + 1] += lv->node_ptr[j];
    lv->node_idx.assign(size_t(ng * npg), 0);
    {
        std::vector<int32_t> fill(lv->node_ptr.begin(), lv->node_ptr.end() - 1);
        for (int64_t e = 0; e < ng * npg; ++e) lv->node_idx[fill[lv->groups[e]]++] = int32_t(e);
    }
    // block sparsity: nodes i, j coupled when they share a group
    std::vector<std::vector<int32_t>> cols(static_cast<size_t>(n));
    for (int64_t g = 0; g < ng; ++g)
        for (int i = 0; i < npg; ++i)
            for (int j = 0; j < npg; ++j) cols[lv->groups[g * npg + i]].push_back(lv->groups[g * npg + j]);
    lv->row_ptr.assign(size_t(n + 1), 0);
    lv->col_idx.clear();
    for (int64_t i = 0; i < n; ++i) {
        auto& c = cols[i];
        std::sort(c.begin(), c.end());
        c.erase(std::unique(c.begin(), c.end()), c.end());
        lv->col_idx.insert(lv->col_idx.end(), c.begin(), c.end());
        lv->row_ptr[i + 1] = int32_t(lv->col_idx.size());
        std::vector<int32_t>().swap(c);
    }
    const int64_t nnzb = int64_t(lv->col_idx.size());
    auto block_of = [&](int32_t i, int32_t j) {
        const int32_t* b = lv->col_idx.data() + lv->row_ptr[i];
        const int32_t* e = lv->col_idx.data() + lv->row_ptr[i + 1];
        return int32_t(std::lower_bound(b, e, j) - lv->col_idx.data());
    };
    lv->grp_blk.assign(size_t(ng * npg * npg), 0);
    std::vector<int32_t> cnt(size_t(nnzb + 1), 0);
    for (int64_t g = 0; g < ng; ++g)
        for (int i = 0; i < npg; ++i)
            for (int j = 0; j < npg; ++j) {
                const int32_t b = block_of(lv->groups[g * npg + i], lv->groups[g * npg + j]);
                lv->grp_blk[size_t((g * npg + i) * npg + j)] = b;
                cnt[b + 1]++;
            }
    for (int64_t b = 0; b < nnzb; ++b) cnt[b + 1] += cnt[b];
    lv->blk_ptr = cnt;
    lv->blk_src.assign(size_t(ng * npg * npg), 0);
    for (int64_t e = 0; e < ng * npg * npg; ++e) lv->blk_src[cnt[lv->grp_blk[e]]++] = int32_t(e);
    // greedy colouring of the groups in group order: the smallest colour that
    // no earlier group sharing a node has
    std::vector<int32_t> color(size_t(ng), -1);
    int ncol = 0;
    std::vector<int64_t> seen_at;   // colour -> last group that marked it
    for (int64_t g = 0; g < ng; ++g) {
        for (int i = 0; i < npg; ++i) {
            const int32_t j = lv->groups[size_t(g * npg + i)];
            for (int32_t e = lv->node_ptr[j]; e < lv->node_ptr[j + 1]; ++e) {
                const int32_t c = color[size_t(lv->node_idx[e] / npg)];
                if (c >= 0) seen_at[size_t(c)] = g;
            }
        }
        int c = 0;
        while (c < ncol && seen_at[size_t(c)] == g) ++c;
        if (c == ncol) {
            ++ncol;
            seen_at.push_back(-1);
        }
        color[size_t(g)] = c;
    }
    lv->color_ptr.assign(size_t(ncol + 1), 0);
    for (int32_t c : color) lv->color_ptr[size_t(c) + 1]++;
    for (int c = 0; c < ncol; ++c) lv->color_ptr[c + 1] += lv->color_ptr[c];
    lv->color_groups.assign(size_t(ng), 0);
    std::vector<int32_t> fill(lv->color_ptr.begin(), lv->color_ptr.end() - 1);
    for (int64_t g = 0; g < ng; ++g) lv->color_groups[size_t(fill[size_t(color[size_t(g)])]++)] = int32_t(g);
}

// A level from cells: grouped (27-node groups, local projection) when its
// cells come in groups of 8 children, else one 8-node "group" per cell.
void level_from_cells(int64_t n, std::vector<double> xyz, std::vector<uint8_t> dir, bool mean_zero,
                      const std::vector<int32_t>& cells, HostLevel* lv) {
    const int64_t nc = int64_t(cells.size() / 8);
    lv->n = n;
    lv->xyz = std::move(xyz);
    lv->dir = std::move(dir);
    lv->mean_zero_pressure = mean_zero;
    std::vector<int32_t> g27;
    if (group_cells(cells, nc, &g27)) {
        lv->ng = nc / 8;
        lv->npg = 27;
        lv->lps = true;
        lv->groups = std::move(g27);
    } else {
        lv->ng = nc;
        lv->npg = 8;
        lv->lps = false;
        lv->groups = cells;
    }
    finish_level(lv);
}

// trilinear weight of parent corner K at group node iota (reference point iota / 2)
double corner_weight(int iota, int K) {
    const int c[3] = {iota % 3, (iota / 3) % 3, iota / 9};
    double w = 1.0;
    for (int d = 0; d < 3; ++d) {
        const double x = 0.5 * c[d];
        w *= ((K >> d) & 1) ? x : 1.0 - x;
    }
    return w;
}

}  // namespace

void build_level(const HostHierarchy& h, bool fine, HostLevel* lv) {
    if (h.element == 2) {
        // Q2 levels: the coarse level's cells are the coarse cells with their
        // 27 level-(L+1) nodes, the fine level's the 8 children of every
        // patch with their 27 level-(L+2) nodes
        const std::vector<int32_t>& kind = fine ? h.kind_f : h.kind_mid;
        lv->q2 = true;
        lv->npg = 27;
        lv->lps = true;
        lv->n = fine ? h.n_fine : h.n_mid;
        lv->xyz = fine ? h.xyz_f : h.xyz_mid;
        lv->dir.resize(size_t(lv->n));
        bool outflow = false;
        for (int64_t j = 0; j < lv->n; ++j) {
            lv->dir[j] = (kind[j] == 1 || kind[j] == 2) ? 1 : 0;
            outflow |= kind[j] == 3;
        }
        lv->mean_zero_pressure = !outflow;
        if (fine) {
            lv->ng = 8 * h.nc;
            lv->groups.resize(size_t(27 * lv->ng));
            for (int64_t P = 0; P < h.nc; ++P)
                for (int t = 0; t < 8; ++t)
                    for (int a = 0; a < 27; ++a) {
                        const int i = t & 1, j = (t >> 1) & 1, k = (t >> 2) & 1;
                        const int iota = (2 * i + a % 3) + 5 * (2 * j + (a / 3) % 3) + 25 * (2 * k + a / 9);
                        lv->groups[size_t(27 * (8 * P + t) + a)] = h.patch_map[size_t(125 * P + iota)];
                    }
        } else {
            lv->ng = h.nc;
            lv->groups = h.patch_map_mid;
        }
        finish_level(lv);
        return;
    }
    if (fine) {
        lv->n = h.n_fine;
        lv->npg = 27;
        lv->lps = true;
        if (h.J == 2) {
            // level L+2: one group per level-(L+1) cell (8 per patch), its 27
            // level-(L+2) nodes taken from the 125-node patch
            lv->ng = 8 * h.nc;
            lv->groups.resize(size_t(27 * lv->ng));
            for (int64_t P = 0; P < h.nc; ++P)
                for (int t = 0; t < 8; ++t)
                    for (int a = 0; a < 27; ++a) {
                        const int i = t & 1, j = (t >> 1) & 1, k = (t >> 2) & 1;
                        const int iota = (2 * i + a % 3) + 5 * (2 * j + (a / 3) % 3) + 25 * (2 * k + a / 9);
                        lv->groups[size_t(27 * (8 * P + t) + a)] = h.patch_map[size_t(125 * P + iota)];
                    }
        } else {
            lv->ng = h.nc;
            lv->groups = h.patch_map;
        }
        lv->xyz = h.xyz_f;
        lv->dir.resize(size_t(h.n_fine));
        bool outflow = false;
        for (int64_t j = 0; j < h.n_fine; ++j) {
            lv->dir[j] = (h.kind_f[j] == 1 || h.kind_f[j] == 2) ? 1 : 0;
            outflow |= h.kind_f[j] == 3;
        }
        lv->mean_zero_pressure = !outflow;
        finish_level(lv);
        return;
    }
    std::vector<uint8_t> dir(size_t(h.nv));
    bool outflow = false;
    for (int64_t v = 0; v < h.nv; ++v) {
        dir[v] = (h.bc_c[v] == 1 || h.bc_c[v] == 2) ? 1 : 0;
        outflow |= h.bc_c[v] == 3;
    }
    level_from_cells(h.nv, h.xyz_c, std::move(dir), !outflow, h.cells, lv);
}

bool coarsen_level(const HostLevel& f, HostLevel* c, MgTransfer* t) {
    if (f.npg != 27 || f.ng == 0 || f.q2) return false;   // Q2 transfer is not the trilinear one
    const int64_t ng = f.ng;
    // parent cells: the 8 corners of each group; they must be the nodes
    // 0 .. nc - 1 of the level (numbered coarsest level first)
    std::vector<int32_t> cells(size_t(8 * ng));
    int32_t nmax = -1;
    for (int64_t g = 0; g < ng; ++g)
        for (int K = 0; K < 8; ++K) {
            const int iota = 2 * (K & 1) + 6 * ((K >> 1) & 1) + 18 * ((K >> 2) & 1);
            const int32_t v = f.groups[size_t(27 * g + iota)];
            cells[size_t(8 * g + K)] = v;
            nmax = std::max(nmax, v);
        }
    const int64_t nc = int64_t(nmax) + 1;
    if (nc >= f.n) return false;
    std::vector<uint8_t> seen(size_t(nc), 0);
    for (int32_t v : cells) seen[size_t(v)] = 1;
    for (uint8_t s : seen)
        if (!s) return false;
    std::vector<double> xyz(f.xyz.begin(), f.xyz.begin() + 3 * nc);
    std::vector<uint8_t> dir(f.dir.begin(), f.dir.begin() + nc);
    // a level with almost no free velocity nodes cannot carry the coarse
    // pressure modes (the continuity rows then see hardly any velocity, and
    // only the stabilisation would fix the pressure): stop above it
    int64_t free_nodes = 0;
    for (uint8_t d : dir) free_nodes += d ? 0 : 1;
    if (free_nodes < kMinFreeCoarseNodes) return false;
    level_from_cells(nc, std::move(xyz), std::move(dir), f.mean_zero_pressure, cells, c);
    // prolongation rows: fine node j takes the trilinear weights of the
    // corners of the first group (in group order) that contains it
    const int64_t n = f.n;
    t->P_ptr.assign(size_t(n + 1), 0);
    t->P_idx.clear();
    t->P_w.clear();
    for (int64_t j = 0; j < n; ++j) {
        const int32_t e = f.node_idx[size_t(f.node_ptr[j])];
        const int64_t g = e / 27;
        const int iota = int(e % 27);
        for (int K = 0; K < 8; ++K) {
            const double w = corner_weight(iota, K);
            if (w == 0.0) continue;
            t->P_idx.push_back(cells[size_t(8 * g + K)]);
            t->P_w.push_back(w);
        }
        t->P_ptr[j + 1] = int32_t(t->P_idx.size());
    }
    // restriction = transpose, rows in increasing fine node order
    t->R_ptr.assign(size_t(nc + 1), 0);
    for (int32_t v : t->P_idx) t->R_ptr[size_t(v) + 1]++;
    for (int64_t i = 0; i < nc; ++i) t->R_ptr[i + 1] += t->R_ptr[i];
    t->R_idx.assign(t->P_idx.size(), 0);
    t->R_w.assign(t->P_idx.size(), 0.0);
    std::vector<int32_t> fill(t->R_ptr.begin(), t->R_ptr.end() - 1);
    for (int64_t j = 0; j < n; ++j)
        for (int32_t e = t->P_ptr[j]; e < t->P_ptr[j + 1]; ++e) {
            const int32_t at = fill[size_t(t->P_idx[e])]++;
            t->R_idx[size_t(at)] = int32_t(j);
            t->R_w[size_t(at)] = t->P_w[size_t(e)];
        }
    return true;
}

}  // namespace dnnmg
