// ec_slice.h -- per-voxel changes of the 3D curves from planar images.
//
// Slicing the closed cubical complex by z (Sec. 2 builds it from the top
// cells: an active voxel brings all its faces, edges and vertices):
//   * a cell that lies in the grid plane z = j is present at level k iff its
//     xy-shadow is in the closed 2D complex of the image m_j = min(b_{j-1}, b_j)
//     (it is incident to the voxels above and below its shadow);
//   * a cell that spans the layer (j, j+1) is present iff its shadow is in the
//     closed 2D complex of the layer image b_j, and it has one dimension more.
// Hence, at every level (Eq. EC_formula counts cells with alternating signs)
//     chi_3D = sum_{j=0..D} chi_2D(m_j) - sum_{j=0..D-1} chi_2D(b_j),
// with b_{-1} = b_D = never active.  Each 2D term is regrouped per pixel as in
// the 2D kernel: ordering the pixels of one image by (level, linear index),
// pixel p brings its face, the edges none of whose other pixel precedes it and
// the corners none of whose 3 other pixels precede it, a change of
// 1 + nE - nV (nE: edge neighbours that precede, nV: corners already covered)
// added at p's level.  A pixel of m_j has the level of the voxel below or
// above it; its change goes to that voxel (the lower one on ties), so every
// voxel c = (x, y, s) makes one histogram update per descriptor:
//   d_EC(c) = -d_{b_s}(x,y) + [b_s < b_{s-1}] d_{m_s}(x,y) + [b_s <= b_{s+1}] d_{m_{s+1}}(x,y).
// Every cell is counted once, at its entry level, so the per-level sums equal
// those of the vertex tables (Tables 1 and 2); only which voxel carries a
// cell can differ from the 26-neighbour form (ec_rules.h) when levels tie.
//
// Surface area and crease perimeter keep the 26-neighbour rules of
// voxel_delta_3d (order (level, linear index)): the in-plane face and diagonal
// comparisons are those of the layer image, the z faces come from the
// comparison of the two planes, and the crease rule of the x and y edges needs
// the four diagonal neighbours across each plane.
//
// Representation: as in ec_swar.h, a thread holds four consecutive voxels of
// a row as two words of 16-bit keys; comparisons of one neighbour offset for
// the four voxels end as one byte mask (byte v = 0xFF iff the neighbour
// precedes voxel v), and sums of byte masks times 255^-1 mod 2^32 count per
// byte.  Row5 holds the five key-pair words of one row around the quad.
#pragma once
#include <stdint.h>

#include "ec_rules.h"
#include "ec_swar.h"

namespace ec {

// Keys (x-1, x), (x, x+1), (x+1, x+2), (x+2, x+3), (x+3, x+4) of one row,
// low lane first.
struct Row5 {
    uint32_t a, b, c, d, e;
};

// Lane-wise minimum of two words of two 16-bit keys.
EC_HD uint32_t vmin2(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
#else
    const uint32_t lo = (a & 0xFFFFu) < (b & 0xFFFFu) ? (a & 0xFFFFu) : (b & 0xFFFFu);
    const uint32_t hi = (a >> 16) < (b >> 16) ? (a >> 16) : (b >> 16);
    return lo | (hi << 16);
#endif
}

EC_HD Row5 vmin_row(const Row5 &p, const Row5 &q)
{
    return Row5{vmin2(p.a, q.a), vmin2(p.b, q.b), vmin2(p.c, q.c), vmin2(p.d, q.d), vmin2(p.e, q.e)};
}

// Comparison words.  For centre pair C and neighbour pair N (lanes < 0x8000),
// lane bit 15 of C + 0x8000 - N - k is [N <= C - k]:
//   EARLIER neighbours (before c in linear order) precede on ties: k = 0;
//   LATER neighbours precede only when strictly smaller: k = 1.
EC_HD uint32_t cmp_earlier(uint32_t c, uint32_t n) { return c + 0x80008000u - n; }
EC_HD uint32_t cmp_later(uint32_t c, uint32_t n) { return c + 0x7FFF7FFFu - n; }

// Byte masks of one planar image around a quad (rows dy = -1, 0, +1).
// fxmc is the COMPLEMENT of the (-1, 0) mask: its bytes 1..3 are the
// (+1, 0) mask's bytes 0..2 (the same pairs seen from the other side) and
// byte 0 comes from one more lane comparison.
struct ImgMasks {
    uint32_t fxmc, fxp, fym, fyp;   // in-plane face (2D edge) neighbours
    uint32_t dmm, dpm, dmp, dpp;    // in-plane diagonals (dx, dy) = (-,-) (+,-) (-,+) (+,+)
};

EC_HD ImgMasks img_masks(const Row5 &m, const Row5 &c, const Row5 &p)
{
    ImgMasks k;
    const uint32_t B = c.b, D = c.d;
    k.dmm = sign_bytes4(cmp_earlier(B, m.a), cmp_earlier(D, m.c));
    k.fym = sign_bytes4(cmp_earlier(B, m.b), cmp_earlier(D, m.d));
    k.dpm = sign_bytes4(cmp_earlier(B, m.c), cmp_earlier(D, m.e));
    k.fxp = sign_bytes4(cmp_later(B, c.c), cmp_later(D, c.e));
    // lane 0 of cmp_later(A, B) is [b_x < b_{x-1}]: not (x-1 precedes x)
#if defined(__CUDA_ARCH__)
    {
        uint32_t d;
        asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(cmp_later(c.a, B)), "r"(k.fxp), "n"(0x6549));
        k.fxmc = d;
    }
#else
    {
        const uint32_t u = cmp_later(c.a, B);
        k.fxmc = ((u >> 15) & 1u ? 0xFFu : 0u) | (k.fxp << 8);
    }
#endif
    k.dmp = sign_bytes4(cmp_later(B, p.a), cmp_later(D, p.c));
    k.fyp = sign_bytes4(cmp_later(B, p.b), cmp_later(D, p.d));
    k.dpp = sign_bytes4(cmp_later(B, p.c), cmp_later(D, p.e));
    return k;
}

// prmt.b32 with an immediate selector (host: the same byte selection).
template <uint32_t SEL>
EC_HD uint32_t prmt_imm(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "n"(SEL));
    return d;
#else
    const uint64_t src = (uint64_t)a | ((uint64_t)b << 32);
    uint32_t d = 0;
    for (int i = 0; i < 4; i++) {
        const uint32_t n = (SEL >> (4 * i)) & 0xFu;
        uint32_t byte = (uint32_t)(src >> (8 * (n & 7u))) & 0xFFu;
        if (n & 8u) byte = (byte & 0x80u) ? 0xFFu : 0u;
        d |= byte << (8 * i);
    }
    return d;
#endif
}

// Masks of two stacked quads of one planar image, rows y (A) and y+1 (B);
// r0..r3 = rows y-1 .. y+2.  The three pairs between the two rows are
// compared once: B's dy = -1 masks are A's dy = +1 masks seen from the
// other side (complements, shifted by one byte for the diagonals), plus one
// lane comparison each for the diagonal pair that leaves the quad.
EC_HD void img_masks2(const Row5 &r0, const Row5 &r1, const Row5 &r2, const Row5 &r3, ImgMasks &A, ImgMasks &B)
{
    A = img_masks(r0, r1, r2);
    const uint32_t Bb = r2.b, Bd = r2.d;
    B.fxp = sign_bytes4(cmp_later(Bb, r2.c), cmp_later(Bd, r2.e));
    B.fxmc = prmt_imm<0x6549>(cmp_later(r2.a, Bb), B.fxp);
    B.dmp = sign_bytes4(cmp_later(Bb, r3.a), cmp_later(Bd, r3.c));
    B.fyp = sign_bytes4(cmp_later(Bb, r3.b), cmp_later(Bd, r3.d));
    B.dpp = sign_bytes4(cmp_later(Bb, r3.c), cmp_later(Bd, r3.e));
    B.fym = ~A.fyp;
    // byte 0: not [(x-1, y) precedes (x, y+1)]; bytes 1..3: A's (+1,+1) bytes 0..2
    B.dmm = ~prmt_imm<0x6549>(cmp_later(r1.a, Bb), A.dpp);
    // bytes 0..2: A's (-1,+1) bytes 1..3; byte 3: not [(x+4, y) precedes (x+3, y+1)]
    B.dpm = ~prmt_imm<0xF321>(A.dmp, cmp_later(r1.e, Bd));
}

// 255 * (nE + 1) per digit (mod 2^32): the face (2D edge) masks summed, with
// the complemented (-1, 0) mask folded in (~f = -1 - f).
EC_HD uint32_t img_sEp1(const ImgMasks &k) { return (k.fxp + k.fym) + (k.fyp - k.fxmc); }

// 255 * (nV - nE) per digit (mod 2^32) from the corner covers and sEp1.
EC_HD uint32_t img_raw(const ImgMasks &k, uint32_t sEp1)
{
    const uint32_t cmm = ~k.fxmc | k.fym | k.dmm, cpm = k.fxp | k.fym | k.dpm;
    const uint32_t cmp = ~k.fxmc | k.fyp | k.dmp, cpp = k.fxp | k.fyp | k.dpp;
    return ((cmm + cpm) + (cmp + cpp)) - sEp1 + 1u;
}

// Signed-byte changes of the four voxels of a quad.
struct SliceOut {
    uint32_t ec, area, per;
};

// What a thread carries from one plane to the next.
struct SliceState {
    uint32_t dm;       // changes of the pixels of m_s, 0x40 + d per byte
    uint32_t z;        // [b_{s-1} <= b_s] per byte: the voxel below precedes
    uint32_t dd[4];    // crease only: [n precedes c] for c in plane s and n its diagonal
                       // neighbours (-1,0,-1) (+1,0,-1) (0,-1,-1) (0,+1,-1)
};

// Changes of the m-image pixels between planes s and s+1 and the masks of the
// z comparison.  P = plane s, Q = plane s+1 (rows dy = -1, 0, +1).
template <bool PER>
EC_HD void slice_upper(const Row5 (&P)[3], const Row5 (&Q)[3], uint32_t &dm_next, uint32_t &z, uint32_t (&dd)[4])
{
    const Row5 m0 = vmin_row(P[0], Q[0]), m1 = vmin_row(P[1], Q[1]), m2 = vmin_row(P[2], Q[2]);
    const ImgMasks km = img_masks(m0, m1, m2);
    // x * 0x01010101 = -x / 255 (mod 2^32): digits 0x40 + 1 + nE - nV
    dm_next = img_raw(km, img_sEp1(km)) * 0x01010101u + 0x41414141u;
    // byte v: [b_s <= b_{s+1}], the voxel of plane s precedes the one above
    z = sign_bytes4(cmp_earlier(Q[1].b, P[1].b), cmp_earlier(Q[1].d, P[1].d));
    if (PER) {
        // voxels of plane s+1 against their diagonal neighbours in plane s
        // (earlier in linear order)
        dd[0] = sign_bytes4(cmp_earlier(Q[1].b, P[1].a), cmp_earlier(Q[1].d, P[1].c));
        dd[1] = sign_bytes4(cmp_earlier(Q[1].b, P[1].c), cmp_earlier(Q[1].d, P[1].e));
        dd[2] = sign_bytes4(cmp_earlier(Q[1].b, P[0].b), cmp_earlier(Q[1].d, P[0].d));
        dd[3] = sign_bytes4(cmp_earlier(Q[1].b, P[2].b), cmp_earlier(Q[1].d, P[2].d));
    }
}

// Start of a z walk: P = plane s0 - 1, Q = plane s0; fills the state for
// counting plane s0.
template <bool PER>
EC_HD void slice_begin(const Row5 (&P)[3], const Row5 (&Q)[3], SliceState &st)
{
    slice_upper<PER>(P, Q, st.dm, st.z, st.dd);
}

// What to produce for the area descriptor.
enum { AREA_NONE = 0, AREA_SIGNED = 1, AREA_FREE_FACES = 2 };

// Changes of one quad of plane s from its layer-image masks kb, the decoded
// m-image changes dm_next of the plane above, the z masks z = [b_s <= b_{s+1}]
// and (crease) the diagonal masks: u = the four diagonals of plane s+1 around
// the quad, dd_next = the diagonal-down masks of the quad above.  Advances st
// to plane s+1.
//   AREA_SIGNED:     o.area = signed-byte area changes 6 - 2 nF;
//   AREA_FREE_FACES: o.area = unsigned bytes 6 - nF (the faces c brings),
//                    from which the area change is 2 (6 - nF) - 6.
template <int AREA, bool PER>
EC_HD SliceOut slice_finish(const ImgMasks &kb, uint32_t dm_next, uint32_t z, const uint32_t (&u)[4],
                            const uint32_t (&dd_next)[4], SliceState &st)
{
    const uint32_t sEp1 = img_sEp1(kb);
    const uint32_t rawb = img_raw(kb, sEp1);
    const uint32_t selA = (st.dm & ~st.z) | (0x40404040u & st.z);
    const uint32_t selB = (dm_next & z) | (0x40404040u & ~z);
    SliceOut o;
    o.ec = (selA + selB - rawb * 0x01010101u - 0x01010101u) ^ 0x80808080u;
    o.area = 0u;
    // faces present: the in-plane ones (sEp1 - 1), the one below (st.z), the
    // one above (~z = -1 - z): 255 nF = sEp1 + st.z - z - 2
    if (AREA == AREA_SIGNED) o.area = ((sEp1 + st.z - z) * 0x02020202u + 0x82828282u) ^ 0x80808080u;
    if (AREA == AREA_FREE_FACES) o.area = (sEp1 + st.z - z) * 0x01010101u + 0x04040404u;
    o.per = 0u;
    if (PER) {
        const uint32_t fxm = ~kb.fxmc, above = ~z, below = st.z;
        const uint32_t s1 = (maj3(fxm, kb.fym, ~kb.dmm) + maj3(kb.fxp, kb.fym, ~kb.dpm)) +
                            (maj3(fxm, kb.fyp, ~kb.dmp) + maj3(kb.fxp, kb.fyp, ~kb.dpp));
        const uint32_t s2 = (maj3(fxm, above, ~u[0]) + maj3(kb.fxp, above, ~u[1])) +
                            (maj3(kb.fym, above, ~u[2]) + maj3(kb.fyp, above, ~u[3]));
        const uint32_t s3 = (maj3(fxm, below, ~st.dd[0]) + maj3(kb.fxp, below, ~st.dd[1])) +
                            (maj3(kb.fym, below, ~st.dd[2]) + maj3(kb.fyp, below, ~st.dd[3]));
        o.per = ((s1 + s2 + s3) * 0x02020202u + 0x8C8C8C8Cu) ^ 0x80808080u;
        st.dd[0] = dd_next[0]; st.dd[1] = dd_next[1]; st.dd[2] = dd_next[2]; st.dd[3] = dd_next[3];
    }
    st.dm = dm_next;
    st.z = z;
    return o;
}

// Decoded m-image changes (0x40 + d per byte) from its masks.
EC_HD uint32_t img_dm(const ImgMasks &km) { return img_raw(km, img_sEp1(km)) * 0x01010101u + 0x41414141u; }

// Crease only: the diagonals (-1,0,+1) (+1,0,+1) (0,-1,+1) (0,+1,+1) of the
// quad with centre pairs (cb, cd) in the plane above (rows q0..q2), later in
// linear order; and the diagonal-down masks of the quad above (centre pairs
// in q1) against this plane's rows p0..p2, earlier in order.
EC_HD void diag_up(uint32_t cb, uint32_t cd, const Row5 &q0, const Row5 &q1, const Row5 &q2, uint32_t (&u)[4])
{
    u[0] = sign_bytes4(cmp_later(cb, q1.a), cmp_later(cd, q1.c));
    u[1] = sign_bytes4(cmp_later(cb, q1.c), cmp_later(cd, q1.e));
    u[2] = sign_bytes4(cmp_later(cb, q0.b), cmp_later(cd, q0.d));
    u[3] = sign_bytes4(cmp_later(cb, q2.b), cmp_later(cd, q2.d));
}
EC_HD void diag_down(const Row5 &q1, const Row5 &p0, const Row5 &p1, const Row5 &p2, uint32_t (&dd)[4])
{
    dd[0] = sign_bytes4(cmp_earlier(q1.b, p1.a), cmp_earlier(q1.d, p1.c));
    dd[1] = sign_bytes4(cmp_earlier(q1.b, p1.c), cmp_earlier(q1.d, p1.e));
    dd[2] = sign_bytes4(cmp_earlier(q1.b, p0.b), cmp_earlier(q1.d, p0.d));
    dd[3] = sign_bytes4(cmp_earlier(q1.b, p2.b), cmp_earlier(q1.d, p2.d));
}

// Two stacked quads (rows y, y+1) of plane s: P, Q = rows y-1 .. y+2 of
// planes s and s+1; sa, sb = the quads' states.
template <int AREA, bool PER>
EC_HD void slice_pair(const Row5 (&P)[4], const Row5 (&Q)[4], SliceState &sa, SliceState &sb, SliceOut &oa,
                      SliceOut &ob)
{
    ImgMasks ka, kb, ma, mb;
    img_masks2(P[0], P[1], P[2], P[3], ka, kb);
    {
        const Row5 m0 = vmin_row(P[0], Q[0]), m1 = vmin_row(P[1], Q[1]);
        const Row5 m2 = vmin_row(P[2], Q[2]), m3 = vmin_row(P[3], Q[3]);
        img_masks2(m0, m1, m2, m3, ma, mb);
    }
    const uint32_t za = sign_bytes4(cmp_earlier(Q[1].b, P[1].b), cmp_earlier(Q[1].d, P[1].d));
    const uint32_t zb = sign_bytes4(cmp_earlier(Q[2].b, P[2].b), cmp_earlier(Q[2].d, P[2].d));
    uint32_t ua[4] = {0u, 0u, 0u, 0u}, ub[4] = {0u, 0u, 0u, 0u}, da[4] = {0u, 0u, 0u, 0u}, db[4] = {0u, 0u, 0u, 0u};
    if (PER) {
        diag_up(P[1].b, P[1].d, Q[0], Q[1], Q[2], ua);
        diag_up(P[2].b, P[2].d, Q[1], Q[2], Q[3], ub);
        diag_down(Q[1], P[0], P[1], P[2], da);
        diag_down(Q[2], P[1], P[2], P[3], db);
    }
    oa = slice_finish<AREA, PER>(ka, img_dm(ma), za, ua, da, sa);
    ob = slice_finish<AREA, PER>(kb, img_dm(mb), zb, ub, db, sb);
}

// Start state of two stacked quads: P = plane s0 - 1, Q = plane s0.
template <bool PER>
EC_HD void slice_pair_begin(const Row5 (&P)[4], const Row5 (&Q)[4], SliceState &sa, SliceState &sb)
{
    const Row5 P3a[3] = {P[0], P[1], P[2]}, Q3a[3] = {Q[0], Q[1], Q[2]};
    const Row5 P3b[3] = {P[1], P[2], P[3]}, Q3b[3] = {Q[1], Q[2], Q[3]};
    slice_upper<PER>(P3a, Q3a, sa.dm, sa.z, sa.dd);
    slice_upper<PER>(P3b, Q3b, sb.dm, sb.z, sb.dd);
}

// Changes of the four voxels of plane s (P) given plane s+1 (Q); advances st
// to plane s+1.
template <bool AREA, bool PER>
EC_HD SliceOut slice_quad(const Row5 (&P)[3], const Row5 (&Q)[3], SliceState &st)
{
    const ImgMasks kb = img_masks(P[0], P[1], P[2]);
    const uint32_t sEp1 = img_sEp1(kb);
    const uint32_t rawb = img_raw(kb, sEp1);
    uint32_t dm_next, z, dd_next[4];
    slice_upper<PER>(P, Q, dm_next, z, dd_next);
    // the voxel owns m_s unless the one below precedes it; it owns m_{s+1}
    // when it precedes the one above.  Unowned bytes read 0x40 (no change).
    const uint32_t selA = (st.dm & ~st.z) | (0x40404040u & st.z);
    const uint32_t selB = (dm_next & z) | (0x40404040u & ~z);
    SliceOut o;
    // digits 0x80 + d_A + d_B - (1 + nE_b - nV_b)
    o.ec = (selA + selB - rawb * 0x01010101u - 0x01010101u) ^ 0x80808080u;
    o.area = 0u;
    if (AREA) {
        // faces present: nE_b in-plane, the voxel below (st.z), the voxel above (~z);
        // area change 6 - 2 nF; sEp1 + st.z + ~z = 255 nF + (1 - 1 - 1) ... folded below
        o.area = ((sEp1 + st.z - z) * 0x02020202u + 0x82828282u) ^ 0x80808080u;
    }
    o.per = 0u;
    if (PER) {
        // crease rule per edge of c: the weight drops iff more of its two face
        // neighbours than its diagonal neighbour precede, maj(a1, a2, ~d)
        const uint32_t fxm = ~kb.fxmc, above = ~z, below = st.z;
        // z edges (in-plane corners)
        uint32_t s1 = (maj3(fxm, kb.fym, ~kb.dmm) + maj3(kb.fxp, kb.fym, ~kb.dpm)) +
                      (maj3(fxm, kb.fyp, ~kb.dmp) + maj3(kb.fxp, kb.fyp, ~kb.dpp));
        // edges in plane s+1: diagonals (-1,0,+1) (+1,0,+1) (0,-1,+1) (0,+1,+1), later in order
        const uint32_t u0 = sign_bytes4(cmp_later(P[1].b, Q[1].a), cmp_later(P[1].d, Q[1].c));
        const uint32_t u1 = sign_bytes4(cmp_later(P[1].b, Q[1].c), cmp_later(P[1].d, Q[1].e));
        const uint32_t u2 = sign_bytes4(cmp_later(P[1].b, Q[0].b), cmp_later(P[1].d, Q[0].d));
        const uint32_t u3 = sign_bytes4(cmp_later(P[1].b, Q[2].b), cmp_later(P[1].d, Q[2].d));
        uint32_t s2 = (maj3(fxm, above, ~u0) + maj3(kb.fxp, above, ~u1)) +
                      (maj3(kb.fym, above, ~u2) + maj3(kb.fyp, above, ~u3));
        // edges in plane s: the diagonals below, computed one plane earlier
        uint32_t s3 = (maj3(fxm, below, ~st.dd[0]) + maj3(kb.fxp, below, ~st.dd[1])) +
                      (maj3(kb.fym, below, ~st.dd[2]) + maj3(kb.fyp, below, ~st.dd[3]));
        o.per = ((s1 + s2 + s3) * 0x02020202u + 0x8C8C8C8Cu) ^ 0x80808080u;
        st.dd[0] = dd_next[0]; st.dd[1] = dd_next[1]; st.dd[2] = dd_next[2]; st.dd[3] = dd_next[3];
    }
    st.dm = dm_next;
    st.z = z;
    return o;
}

}  // namespace ec
