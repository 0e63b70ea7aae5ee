// Dual medial mesh of the restricted power diagram and its thinning.
//
// Sec. 3.2: the medial mesh is the dual of the RPD: one vertex per sphere with
// a nonempty restricted power cell, an edge (i, j) per RPF, a triangle
// (i, j, k) per RPE and a tetrahedron (i, j, k, l) per RPV.
//
// Sec. 5.3 (geometry-guided thinning): a simple pair (x, y) is a simplex x and
// a face y of x that no other simplex of the complex has as a face; removing
// it keeps the complex's homotopy type.  Every triangle f_ijk gets the
// importance alpha_ijk = length(RPE_ijk) / mean(2 r_i, 2 r_j, 2 r_k).  First
// the tet-face simple pairs are removed, least important triangle first, until
// no tetrahedron is left; then the triangle-edge simple pairs whose triangle
// belonged to an original tetrahedron are removed, least important first,
// while the importance is below sigma.
//
// Ties (readings of the paper, which does not fix them): equal importances go
// to the triangle whose key (sorted sphere ids) is lexicographically
// smallest; a triangle with several free edges gives up the edge with the
// smallest key.  Runs on the host: the pruning is a sequential priority
// process over a complex of a few 10^4 simplices.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <set>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace {

using Key3 = std::array<int32_t, 3>;
using Key2 = std::array<int32_t, 2>;

}  // namespace

int medial_thin(const std::vector<int32_t>& edges, const std::vector<int32_t>& faces,
                const std::vector<double>& alpha, const std::vector<int32_t>& tets, double sigma,
                std::vector<uint8_t>& edge_alive, std::vector<uint8_t>& face_alive, std::vector<uint8_t>& tet_alive) {
    const size_t ne = edges.size() / 2, nf = faces.size() / 3, nt = tets.size() / 4;
    edge_alive.assign(ne, 1);
    face_alive.assign(nf, 1);
    tet_alive.assign(nt, 1);
    std::map<Key2, size_t> eid;
    for (size_t e = 0; e < ne; e++) eid[{edges[2 * e], edges[2 * e + 1]}] = e;
    std::map<Key3, size_t> fid;
    for (size_t f = 0; f < nf; f++) fid[{faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]}] = f;
    // boundary relations (keys are sorted, so sub-keys are too)
    std::vector<std::array<long long, 3>> f_edges(nf);
    std::vector<std::array<long long, 4>> t_faces(nt);
    std::vector<int> face_tets(nf, 0), edge_faces(ne, 0);
    std::vector<std::vector<size_t>> face_tet_list(nf), edge_face_list(ne);
    for (size_t f = 0; f < nf; f++) {
        const int32_t* k = &faces[3 * f];
        const Key2 sub[3] = {{k[0], k[1]}, {k[0], k[2]}, {k[1], k[2]}};
        for (int q = 0; q < 3; q++) {
            auto it = eid.find(sub[q]);
            f_edges[f][q] = it == eid.end() ? -1 : (long long)it->second;
            if (it != eid.end()) {
                edge_faces[it->second]++;
                edge_face_list[it->second].push_back(f);
            }
        }
    }
    std::vector<uint8_t> orig(nf, 0);
    for (size_t t = 0; t < nt; t++) {
        const int32_t* k = &tets[4 * t];
        const Key3 sub[4] = {{k[0], k[1], k[2]}, {k[0], k[1], k[3]}, {k[0], k[2], k[3]}, {k[1], k[2], k[3]}};
        for (int q = 0; q < 4; q++) {
            auto it = fid.find(sub[q]);
            t_faces[t][q] = it == fid.end() ? -1 : (long long)it->second;
            if (it != fid.end()) {
                face_tets[it->second]++;
                face_tet_list[it->second].push_back(t);
                orig[it->second] = 1;
            }
        }
    }
    // priority: (alpha, face index); face indices follow key order
    using Item = std::pair<double, size_t>;
    std::set<Item> queue;
    auto push_tf = [&](size_t f) {
        if (face_alive[f] && face_tets[f] == 1) queue.insert({alpha[f], f});
    };
    for (size_t f = 0; f < nf; f++) push_tf(f);
    long long left = (long long)nt;
    while (left > 0 && !queue.empty()) {
        const Item it = *queue.begin();
        queue.erase(queue.begin());
        const size_t f = it.second;
        if (!face_alive[f] || face_tets[f] != 1) continue;
        size_t t = (size_t)-1;
        for (size_t q : face_tet_list[f])
            if (tet_alive[q]) t = q;
        if (t == (size_t)-1) continue;
        tet_alive[t] = 0;
        left--;
        face_alive[f] = 0;
        for (int q = 0; q < 3; q++)
            if (f_edges[f][q] >= 0) edge_faces[f_edges[f][q]]--;
        for (int q = 0; q < 4; q++) {
            const long long g = t_faces[t][q];
            if (g < 0 || (size_t)g == f) continue;
            face_tets[g]--;
            push_tf((size_t)g);
        }
    }
    // triangle-edge pairs of the original tetrahedra's triangles, alpha < sigma
    std::set<Item> q2;
    auto push_fe = [&](size_t f) {
        if (!face_alive[f] || !orig[f] || face_tets[f] != 0 || !(alpha[f] < sigma)) return;
        for (int q = 0; q < 3; q++) {
            const long long e = f_edges[f][q];
            if (e >= 0 && edge_alive[e] && edge_faces[e] == 1) {
                q2.insert({alpha[f], f});
                return;
            }
        }
    };
    for (size_t f = 0; f < nf; f++) push_fe(f);
    while (!q2.empty()) {
        const Item it = *q2.begin();
        q2.erase(q2.begin());
        const size_t f = it.second;
        if (!face_alive[f] || face_tets[f] != 0) continue;
        long long ebest = -1;
        for (int q = 0; q < 3; q++) {   // sub-keys in order: the first free edge has the smallest key
            const long long e = f_edges[f][q];
            if (e >= 0 && edge_alive[e] && edge_faces[e] == 1) {
                ebest = e;
                break;
            }
        }
        if (ebest < 0) continue;
        face_alive[f] = 0;
        edge_alive[ebest] = 0;
        for (int q = 0; q < 3; q++) {
            const long long e = f_edges[f][q];
            if (e < 0 || e == ebest) continue;
            edge_faces[e]--;
            // the other triangle on this edge may have become prunable
            if (edge_faces[e] == 1)
                for (size_t g : edge_face_list[e]) push_fe(g);
        }
    }
    return 0;
}
