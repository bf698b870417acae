// ec_rules.h -- vertex-contribution tables and per-top-cell closed forms.
//
// Vertex contributions (Sec. 2, Table 1 for 2D, Table 2 for 3D): a grid vertex
// owns 1/2 of each incident edge, 1/4 of each incident face and 1/8 of each
// incident voxel.  Its contribution to a descriptor is a function of which
// top cells of its 2x2 (2D) / 2x2x2 (3D) neighbourhood are active.  The tables
// here are derived from that rule, not transcribed; the tests check them
// against the printed tables.  Integer scales make every entry exact:
//   2D: {4*EC(8-C), 4*EC(4-C), 2*perimeter, 4*area}
//   3D: {8*EC(26-C), 2*perimeter(crease), 4*area, 8*volume}
// Mask bits: 2D bit x + 2y, 3D bit x + 2y + 4z, for the neighbourhood cell at
// offset (x, y[, z]) in {0,1}^n from the vertex's lower corner.
//
// Per-top-cell regrouping ("entering cell" form): ordering top cells by
// (level, linear index) makes the filtration add one top cell at a time.  When
// cell c enters, each of its 2^n corner vertices changes type from m to m|c,
// so the total change is sum over corners of T[m|c] - T[m].  Summed over all
// cells this telescopes to the per-vertex sums of Algorithms 1-3, so adding
// that change at c's level gives identical curves with one histogram update
// per top cell.  The closed forms below evaluate that sum from the set of
// neighbours that precede c, by counting the faces, edges and vertices of c's
// closure that c brings in; ec_selfcheck_rules() compares both forms on every
// precedence pattern.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define EC_HD __host__ __device__ __forceinline__
#else
#define EC_HD inline
#endif

namespace ec {

EC_HD int popc32(uint32_t v)
{
#if defined(__CUDA_ARCH__)
    return __popc(v);
#else
    return __builtin_popcount(v);
#endif
}

// ---------------------------------------------------------------- tables

struct Table2D { int32_t v[16][4]; };
struct Table3D { int32_t v[256][4]; };

// Crease weight of an edge from its 4 surrounding top cells, cells numbered
// a + 2b over the two axes perpendicular to the edge: one active -> 1, two
// sharing a face -> 0, two diagonal -> 2, three -> 1, none or four -> 0.
constexpr int crease4(unsigned q)
{
    int n = (int)(q & 1) + (int)(q >> 1 & 1) + (int)(q >> 2 & 1) + (int)(q >> 3 & 1);
    if (n == 1 || n == 3) return 1;
    if (n == 2) return (q == 0x9u || q == 0x6u) ? 2 : 0;
    return 0;
}

constexpr int popc_c(unsigned m)
{
    int n = 0;
    for (int i = 0; i < 8; i++) n += (int)(m >> i & 1);
    return n;
}

constexpr Table2D make_table_2d()
{
    Table2D t{};
    for (unsigned m = 0; m < 16; m++) {
        int V8 = m ? 1 : 0;
        int V4 = V8 + ((m == 0x9u || m == 0x6u) ? 1 : 0);   // diagonal pair: two vertices under 4-C
        int halfE = 0, bnd = 0;
        for (int axis = 0; axis < 2; axis++)
            for (int side = 0; side < 2; side++) {
                // the half-edge leaving the vertex along +/- axis is shared by the
                // two pixels whose coordinate along `axis` equals `side`
                int n = 0;
                for (unsigned b = 0; b < 4; b++)
                    if (((b >> axis) & 1u) == (unsigned)side) n += (int)(m >> b & 1);
                halfE += n > 0 ? 1 : 0;
                bnd += n == 1 ? 1 : 0;
            }
        int F = popc_c(m);
        t.v[m][0] = 4 * V8 - 2 * halfE + F;
        t.v[m][1] = 4 * V4 - 2 * halfE + F;
        t.v[m][2] = bnd;
        t.v[m][3] = F;
    }
    return t;
}

constexpr Table3D make_table_3d()
{
    Table3D t{};
    for (unsigned m = 0; m < 256; m++) {
        int V = m ? 1 : 0;
        int halfE = 0, crease = 0, quarterF = 0, bndF = 0;
        for (int axis = 0; axis < 3; axis++) {
            int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
            for (int side = 0; side < 2; side++) {
                // half-edge along +/- axis: its 4 surrounding voxels have
                // coordinate `side` on `axis`; cross-section index a + 2b
                unsigned q = 0;
                for (unsigned b = 0; b < 8; b++)
                    if (((b >> axis) & 1u) == (unsigned)side && (m >> b & 1u))
                        q |= 1u << (((b >> a1) & 1u) | (((b >> a2) & 1u) << 1));
                halfE += q ? 1 : 0;
                crease += crease4(q);
            }
            // quarter faces normal to `axis`: one per quadrant of (a1, a2);
            // each lies between the two voxels that differ only along `axis`
            for (unsigned s1 = 0; s1 < 2; s1++)
                for (unsigned s2 = 0; s2 < 2; s2++) {
                    int n = 0;
                    for (unsigned s0 = 0; s0 < 2; s0++) {
                        unsigned b = (s0 << axis) | (s1 << a1) | (s2 << a2);
                        n += (int)(m >> b & 1u);
                    }
                    quarterF += n > 0 ? 1 : 0;
                    bndF += n == 1 ? 1 : 0;
                }
        }
        int C = popc_c(m);
        t.v[m][0] = 8 * V - 4 * halfE + 2 * quarterF - C;
        t.v[m][1] = crease;
        t.v[m][2] = bndF;
        t.v[m][3] = C;
    }
    return t;
}

// 3D EC under 6-connectivity, per vertex, scaled by 8.  Under face adjacency
// a cell of the grid belongs to the complex exactly when ALL its incident
// voxels are active (the dual of the closed complex above, whose cells need
// only one), and chi6 = #voxels - #cells of dimension 2 + #dim 1 - #dim 0
// counted over those cells.  A vertex owns 1/8 of each incident voxel, 1/4 of
// each incident face, 1/2 of each incident edge and itself.
struct Table3D6 { int32_t v[256]; };

constexpr Table3D6 make_table_3d_ec6()
{
    Table3D6 t{};
    for (unsigned m = 0; m < 256; m++) {
        int faces = 0, edges = 0;
        for (int axis = 0; axis < 3; axis++) {
            const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
            // quarter faces normal to `axis`: both voxels of the pair active
            for (unsigned s1 = 0; s1 < 2; s1++)
                for (unsigned s2 = 0; s2 < 2; s2++) {
                    const unsigned b0 = (s1 << a1) | (s2 << a2), b1 = b0 | (1u << axis);
                    faces += ((m >> b0) & 1u) && ((m >> b1) & 1u) ? 1 : 0;
                }
            // half edges along `axis`: all four voxels on that side active
            for (unsigned side = 0; side < 2; side++) {
                bool all = true;
                for (unsigned b = 0; b < 8; b++)
                    if (((b >> axis) & 1u) == side && !((m >> b) & 1u)) all = false;
                edges += all ? 1 : 0;
            }
        }
        t.v[m] = popc_c(m) - 2 * faces + 4 * edges - (m == 0xFFu ? 8 : 0);
    }
    return t;
}

// ------------------------------------------------- per-top-cell closed forms

// 3D: P holds one bit per neighbour n of the entering voxel c, set when n
// precedes c; bit (dx+1) + 3*(dy+1) + 9*(dz+1) for offset (dx,dy,dz), the
// centre bit 13 is zero.  Outputs the unscaled changes of EC, crease
// perimeter, boundary area (volume always changes by 1).
//   EC:  c brings itself (-1), each face whose neighbour does not precede (+1),
//        each edge none of whose 3 other voxels precede (-1) and each corner
//        none of whose 7 other voxels precede (+1).
//   area: each face turns from interior-free to boundary (+1) or from
//        boundary to interior (-1, neighbour already active).
//   perimeter: each edge of c changes weight by +1 or -1: -1 exactly when
//        more of c's two face neighbours around it precede than its diagonal
//        neighbour does (alpha > delta with alpha in {0,1,2}, delta in {0,1}).
struct Delta3 { int ec, per, area; };

constexpr uint32_t kFaceMask3 = (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
constexpr uint32_t kEdgeMask3 = 0x2AAAAAAu & ~(1u << 13);   // the 12 neighbours sharing only an edge
constexpr uint32_t kCornerOrigins3 = 0x361Bu;               // {0,1,3,4,9,10,12,13}

EC_HD Delta3 voxel_delta_3d(uint32_t P)
{
    const int nF = popc32(P & kFaceMask3);
    // corner cover: OR of each 2x2x2 block of the 3x3x3 neighbourhood; the
    // block anchored at (vx,vy,vz) in {0,1}^3 is the octant of c's corner.
    uint32_t w1 = P | (P >> 1);
    uint32_t w2 = w1 | (w1 >> 3);
    uint32_t w3 = w2 | (w2 >> 9);
    const int nV = popc32(w3 & kCornerOrigins3);
    // For every edge of c, align its two face neighbours (A1, A2) with the bit
    // of its edge neighbour d: the edge neighbour at offset e has its face
    // neighbours at e with one non-zero coordinate cleared.
    //   z-edges (d at dz=0): A1 = x-face (shift by 3 in y), A2 = y-face (shift by 1 in x)
    //   x-edges (d at dx=0): A1 = y-face (shift by 9 in z), A2 = z-face (shift by 3 in y)
    //   y-edges (d at dy=0): A1 = x-face (shift by 9 in z), A2 = z-face (shift by 1 in x)
    // For a d bit at lower side of an axis the face bit sits one step up that
    // axis (shift right), on the upper side one step down (shift left).
    const uint32_t Pr1 = P >> 1, Pl1 = P << 1, Pr3 = P >> 3, Pl3 = P << 3, Pr9 = P >> 9, Pl9 = P << 9;
    // d positions: z-edges {9,11,15,17}, x-edges {1,7,19,25}, y-edges {3,5,21,23}
    const uint32_t dy_lo_z = (1u << 9) | (1u << 11), dy_hi_z = (1u << 15) | (1u << 17);
    const uint32_t dz_lo = (1u << 1) | (1u << 7) | (1u << 3) | (1u << 5);
    const uint32_t dz_hi = (1u << 19) | (1u << 25) | (1u << 21) | (1u << 23);
    uint32_t A1 = (Pr3 & dy_lo_z) | (Pl3 & dy_hi_z) | (Pr9 & dz_lo) | (Pl9 & dz_hi);
    const uint32_t dx_lo = (1u << 9) | (1u << 15) | (1u << 3) | (1u << 21);
    const uint32_t dx_hi = (1u << 11) | (1u << 17) | (1u << 5) | (1u << 23);
    const uint32_t dy_lo_x = (1u << 1) | (1u << 19), dy_hi_x = (1u << 7) | (1u << 25);
    uint32_t A2 = (Pr1 & dx_lo) | (Pl1 & dx_hi) | (Pr3 & dy_lo_x) | (Pl3 & dy_hi_x);
    const uint32_t cover = (A1 | A2 | P) & kEdgeMask3;
    const uint32_t minus = ((A1 & A2) | ((A1 | A2) & ~P)) & kEdgeMask3;
    const int nE = popc32(cover);
    const int nM = popc32(minus);
    Delta3 d;
    d.ec = 1 - nF + nE - nV;
    d.per = 12 - 2 * nM;
    d.area = 6 - 2 * nF;
    return d;
}

// 3D EC change under 6-connectivity when voxel c enters (P as above): c
// brings itself (+1), completes each face whose neighbour precedes (-1), each
// edge all 3 of whose other voxels precede (+1) and each corner all 7 of
// whose other voxels precede (-1): the AND counterparts of the covers above.
EC_HD int voxel_delta_3d6(uint32_t P)
{
    const int nF = popc32(P & kFaceMask3);
    // corner blocks: AND over each 2x2x2 block with c's own bit set
    const uint32_t Pc = P | (1u << 13);
    const uint32_t w1 = Pc & (Pc >> 1), w2 = w1 & (w1 >> 3), w3 = w2 & (w2 >> 9);
    const int nV = popc32(w3 & kCornerOrigins3);
    // edges: the edge neighbour d and its two face neighbours, aligned at d's
    // bit as in voxel_delta_3d
    const uint32_t Pr1 = P >> 1, Pl1 = P << 1, Pr3 = P >> 3, Pl3 = P << 3, Pr9 = P >> 9, Pl9 = P << 9;
    const uint32_t dy_lo_z = (1u << 9) | (1u << 11), dy_hi_z = (1u << 15) | (1u << 17);
    const uint32_t dz_lo = (1u << 1) | (1u << 7) | (1u << 3) | (1u << 5);
    const uint32_t dz_hi = (1u << 19) | (1u << 25) | (1u << 21) | (1u << 23);
    const uint32_t A1 = (Pr3 & dy_lo_z) | (Pl3 & dy_hi_z) | (Pr9 & dz_lo) | (Pl9 & dz_hi);
    const uint32_t dx_lo = (1u << 9) | (1u << 15) | (1u << 3) | (1u << 21);
    const uint32_t dx_hi = (1u << 11) | (1u << 17) | (1u << 5) | (1u << 23);
    const uint32_t dy_lo_x = (1u << 1) | (1u << 19), dy_hi_x = (1u << 7) | (1u << 25);
    const uint32_t A2 = (Pr1 & dx_lo) | (Pl1 & dx_hi) | (Pr3 & dy_lo_x) | (Pl3 & dy_hi_x);
    const int nE = popc32(A1 & A2 & P & kEdgeMask3);
    return 1 - nF + nE - nV;
}

// 2D: P bit (dx+1) + 3*(dy+1), centre bit 4 zero.  Changes of EC under 8-
// and 4-connectivity, perimeter (area always changes by 1).
//   EC(8-C): +1 (pixel) - new edges + new corners.
//   EC(4-C): EC(8-C) plus the change in the number of corners of type QD
//            (Table 1: a diagonal pair counts two vertices under 4-C): a
//            corner becomes QD when only its diagonal neighbour precedes, and
//            stops being QD when exactly its two edge neighbours precede.
struct Delta2 { int ec8, ec4, per; };

EC_HD Delta2 pixel_delta_2d(uint32_t P)
{
    const int nE = popc32(P & 0xAAu);                   // bits 1,3,5,7
    const uint32_t w1 = P | (P >> 1);
    const uint32_t w2 = w1 | (w1 >> 3);
    const int nV = popc32(w2 & 0x1Bu);                  // corners anchored at {0,1,3,4}
    int qd = 0;
#pragma unroll
    for (int v = 0; v < 4; v++) {
        const int vx = v & 1, vy = v >> 1;
        const uint32_t a1 = (P >> (2 * vx + 3)) & 1u;   // edge neighbour along x
        const uint32_t a2 = (P >> (1 + 6 * vy)) & 1u;   // edge neighbour along y
        const uint32_t dg = (P >> (2 * vx + 6 * vy)) & 1u;
        qd += (int)(dg & ~a1 & ~a2 & 1u) - (int)(a1 & a2 & ~dg & 1u);
    }
    Delta2 d;
    d.ec8 = 1 + nE - nV;
    d.ec4 = d.ec8 + qd;
    d.per = 4 - 2 * nE;
    return d;
}

}  // namespace ec
