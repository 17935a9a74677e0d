// Marching-cubes case table, generated at start-up from a face rule.
//
// Sec. III-B extracts the isosurface A = L "using the marching cubes
// algorithm [35]" and prints no table, so the table is built from a rule:
//
// Numbering: corner b at (b & 1, (b >> 1) & 1, (b >> 2) & 1); edge
// e = 4 a + c_u + 2 c_v runs along axis a at coordinates (c_u, c_v) on the
// other two axes in increasing order.  Bit b of a case is 1 ("inside") when
// A >= L at corner b.
//
// Rule, per cube face, walking its corners counter-clockwise as seen from
// outside the cube: every maximal run of inside corners c_i .. c_j is cut off
// by one directed segment from the face edge entering the run (c_{i-1}, c_i)
// to the face edge leaving it (c_j, c_{j+1}).  A face whose inside corners sit
// on a diagonal therefore gets two segments, one per inside corner, which
// keeps the inside corners apart.  The directed segments chain into closed
// loops (each crossed edge has one segment in and one out); loops are listed
// by their smallest edge id and walked from it.  A loop is fanned into
// triangles from the first vertex, in loop order, whose fan has no diagonal
// between two edges of one common face (that diagonal would lie in the face
// and also belong to the neighbouring cube's fan).  The segment direction
// makes triangle normals (right-hand rule) point from inside to outside.
// Decisions depend only on a face's own four bits, so adjacent cubes agree.
#include <string.h>

#include "ftr_internal.h"

namespace ftr {
namespace {

struct Face {
    int corner[4];   // counter-clockwise seen from outside
    int edge[4];     // edge[i] joins corner[i] and corner[i + 1]
};

int corner_index(int x, int y, int z) { return x | (y << 1) | (z << 2); }

int edge_index(int ca, int cb) {
    const int diff = ca ^ cb;             // one bit: the axis
    const int axis = diff == 1 ? 0 : (diff == 2 ? 1 : 2);
    const int lo = ca < cb ? ca : cb;
    const int p[3] = {lo & 1, (lo >> 1) & 1, (lo >> 2) & 1};
    int u = -1, v = -1;
    for (int c = 0; c < 3; ++c) {
        if (c == axis) continue;
        if (u < 0) u = c; else v = c;
    }
    return 4 * axis + p[u] + 2 * p[v];
}

void build_faces(Face faces[6]) {
    int k = 0;
    for (int a = 0; a < 3; ++a) {
        const int u = (a + 1) % 3, v = (a + 2) % 3;   // e_u x e_v = e_a
        for (int side = 0; side < 2; ++side) {
            // (u, v) coordinates of the corners, counter-clockwise seen from
            // the outward normal (+a for side 1, -a for side 0)
            static const int ccw_pos[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
            static const int ccw_neg[4][2] = {{0, 0}, {0, 1}, {1, 1}, {1, 0}};
            for (int i = 0; i < 4; ++i) {
                const int* uv = side ? ccw_pos[i] : ccw_neg[i];
                int p[3];
                p[a] = side;
                p[u] = uv[0];
                p[v] = uv[1];
                faces[k].corner[i] = corner_index(p[0], p[1], p[2]);
            }
            for (int i = 0; i < 4; ++i)
                faces[k].edge[i] = edge_index(faces[k].corner[i], faces[k].corner[(i + 1) & 3]);
            ++k;
        }
    }
}

// bitmask of the two faces containing each edge
void build_edge_faces(const Face faces[6], int ef[12]) {
    for (int e = 0; e < 12; ++e) ef[e] = 0;
    for (int f = 0; f < 6; ++f)
        for (int i = 0; i < 4; ++i) ef[faces[f].edge[i]] |= 1 << f;
}

}  // namespace

void mc_generate_table(int32_t ntri[256], int32_t tris[256 * kMaxTrisPerCase * 3]) {
    Face faces[6];
    build_faces(faces);
    int ef[12];
    build_edge_faces(faces, ef);
    for (int i = 0; i < 256 * kMaxTrisPerCase * 3; ++i) tris[i] = -1;
    for (int cs = 0; cs < 256; ++cs) {
        int next[12];
        for (int e = 0; e < 12; ++e) next[e] = -1;
        for (int f = 0; f < 6; ++f) {
            int bit[4];
            for (int i = 0; i < 4; ++i) bit[i] = (cs >> faces[f].corner[i]) & 1;
            for (int i = 0; i < 4; ++i) {
                // a run of inside corners starts at i
                if (!bit[i] || bit[(i + 3) & 3]) continue;
                int j = i;
                while (bit[(j + 1) & 3]) j = (j + 1) & 3;
                const int e_in = faces[f].edge[(i + 3) & 3];
                const int e_out = faces[f].edge[j];
                next[e_in] = e_out;
            }
        }
        int nt = 0;
        bool seen[12] = {};
        for (int e0 = 0; e0 < 12; ++e0) {
            if (next[e0] < 0 || seen[e0]) continue;
            int loop[12];
            int m = 0;
            int e = e0;
            do {
                seen[e] = true;
                loop[m++] = e;
                e = next[e];
            } while (e != e0 && m < 12);
            int s = 0;
            for (; s < m; ++s) {
                bool ok = true;
                for (int i = 2; i < m - 1; ++i)
                    if (ef[loop[s]] & ef[loop[(s + i) % m]]) ok = false;
                if (ok) break;
            }
            if (s == m) s = 0;
            for (int i = 1; i + 1 < m; ++i) {
                if (nt < kMaxTrisPerCase) {
                    int32_t* t = tris + (cs * kMaxTrisPerCase + nt) * 3;
                    t[0] = loop[s];
                    t[1] = loop[(s + i) % m];
                    t[2] = loop[(s + i + 1) % m];
                }
                ++nt;
            }
        }
        ntri[cs] = nt;
    }
}

}  // namespace ftr
