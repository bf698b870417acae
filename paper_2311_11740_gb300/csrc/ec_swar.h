// ec_swar.h -- per-voxel contribution changes for four voxels at once.
//
// The regrouped per-top-cell form of Algorithm 3 needs, for every voxel c,
// which of its 26 neighbours precede it in the (level, linear index) order.
// Keys (levels) are at most 15 bits here, so two voxels that are neighbours
// along x share one 32-bit word (lane 0 = bits 0..15, lane 1 = bits 16..31)
// and one subtraction compares both:
//     (C | 0x80008000) - N - k      bit 15 / 31 = [key_n <= key_c - k]
// with k = 0 for neighbours earlier in linear order (ties precede) and k = 1
// for later ones.  No borrow crosses the lanes because C's lane carries
// 0x8000 and N's lane is below 0x8000.
//
// A thread holds four consecutive voxels of a row as two such words.  One
// `prmt` with sign replication turns the two comparison words of a
// neighbour offset into a byte mask: byte v = 0xFF iff that neighbour
// precedes voxel v.  The contribution change then follows from which faces,
// edges and vertices of c's closure are already present (see voxel_delta_3d
// in ec_rules.h), computed bytewise for the four voxels at once:
//   edge covers   (12): an edge of c is present iff one of its 3 other voxels precedes
//   corner covers  (8): a vertex of c is present iff one of its 7 other voxels precedes
//   face bits      (6): a face of c is present iff the voxel across it precedes
//   crease minus  (12): the edge weight drops iff more face neighbours than
//                       diagonal neighbours around it precede (majority of a1, a2, not d)
// Counting: a byte mask word with n_v in {0, 1} per byte equals
// 255 * sum_v n_v 256^v, so adding such words as 32-bit integers (mod 2^32)
// and multiplying by the inverse of 255 modulo 2^32 (= -0x01010101) gives
// sum_v N_v 256^v for the per-voxel counts N_v exactly.  Adding 128 + a
// bias to every byte keeps each digit in [0, 255] (no borrow between bytes),
// and XOR 0x80 leaves each voxel's change as a signed byte.
#pragma once
#include <stdint.h>

#include "ec_rules.h"

namespace ec {

// prmt.b32 in its default mode with all four selector nibbles asking for
// sign replication: output byte v = msb of (a.byte1, a.byte3, b.byte1,
// b.byte3) replicated over 8 bits, i.e. the comparison bits of voxels
// 0, 1 (word a) and 2, 3 (word b).
EC_HD uint32_t sign_bytes4(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(0xFDB9u));
    return d;
#else
    const uint32_t m0 = (a >> 15) & 1u ? 0xFFu : 0u;
    const uint32_t m1 = (a >> 31) & 1u ? 0xFFu : 0u;
    const uint32_t m2 = (b >> 15) & 1u ? 0xFFu : 0u;
    const uint32_t m3 = (b >> 31) & 1u ? 0xFFu : 0u;
    return m0 | (m1 << 8) | (m2 << 16) | (m3 << 24);
#endif
}

// Byte v of w as a signed integer (prmt with sign replication of byte v
// into bytes 1-3).
template <int V>
EC_HD int sbyte(uint32_t w)
{
#if defined(__CUDA_ARCH__)
    // (inline prmt: the __byte_perm intrinsic ignores the sign-replication bit)
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(w), "r"(0u), "n"(V | ((V | 8) << 4) | ((V | 8) << 8) | ((V | 8) << 12)));
    return (int)d;
#else
    return (int)(int8_t)(uint8_t)(w >> (8 * V));
#endif
}

EC_HD uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (a & c) | (b & c); }

// Changes of the four voxels as signed bytes (byte v = voxel v).
struct QuadDelta {
    uint32_t ec, per, area;
};

// n0/n1[(dx+1) + 3*(dy+1) + 9*(dz+1)]: neighbour key pairs of the voxel
// pairs (0, 1) and (2, 3) (every voxel shifted by the same offset); c0, c1:
// the centre key pairs.
template <bool PER>
EC_HD QuadDelta quad_delta(const uint32_t (&n0)[27], uint32_t c0, const uint32_t (&n1)[27], uint32_t c1)
{
    const uint32_t cm0 = c0 | 0x80008000u, cm1 = c1 | 0x80008000u;
    uint32_t b[27];
#pragma unroll
    for (int i = 0; i < 27; i++) {
        const uint32_t k = i > 13 ? 0x00010001u : 0u;
        b[i] = (i == 13) ? 0u : sign_bytes4(cm0 - n0[i] - k, cm1 - n1[i] - k);
    }
#define ECB(dx, dy, dz) b[((dx) + 1) + 3 * ((dy) + 1) + 9 * ((dz) + 1)]
    const uint32_t fxm = ECB(-1, 0, 0), fxp = ECB(1, 0, 0);
    const uint32_t fym = ECB(0, -1, 0), fyp = ECB(0, 1, 0);
    const uint32_t fzm = ECB(0, 0, -1), fzp = ECB(0, 0, 1);
    // edge covers, named by the signs of the two offsets that are non-zero
    const uint32_t zc_mm = fxm | fym | ECB(-1, -1, 0), zc_pm = fxp | fym | ECB(1, -1, 0);
    const uint32_t zc_mp = fxm | fyp | ECB(-1, 1, 0), zc_pp = fxp | fyp | ECB(1, 1, 0);
    const uint32_t xc_mm = fym | fzm | ECB(0, -1, -1), xc_pm = fyp | fzm | ECB(0, 1, -1);
    const uint32_t xc_mp = fym | fzp | ECB(0, -1, 1), xc_pp = fyp | fzp | ECB(0, 1, 1);
    const uint32_t yc_mm = fxm | fzm | ECB(-1, 0, -1), yc_pm = fxp | fzm | ECB(1, 0, -1);
    const uint32_t yc_mp = fxm | fzp | ECB(-1, 0, 1), yc_pp = fxp | fzp | ECB(1, 0, 1);
    // corner covers: the vertex (sx, sy, sz) of c
#define VC(sx, sy, sz, zc, xc, yc) ((zc) | (xc) | (yc) | ECB(sx, sy, sz))
    const uint32_t v_mmm = VC(-1, -1, -1, zc_mm, xc_mm, yc_mm), v_pmm = VC(1, -1, -1, zc_pm, xc_mm, yc_pm);
    const uint32_t v_mpm = VC(-1, 1, -1, zc_mp, xc_pm, yc_mm), v_ppm = VC(1, 1, -1, zc_pp, xc_pm, yc_pm);
    const uint32_t v_mmp = VC(-1, -1, 1, zc_mm, xc_mp, yc_mp), v_pmp = VC(1, -1, 1, zc_pm, xc_mp, yc_pp);
    const uint32_t v_mpp = VC(-1, 1, 1, zc_mp, xc_pp, yc_mp), v_ppp = VC(1, 1, 1, zc_pp, xc_pp, yc_pp);
#undef VC
    // byte-mask sums (each = 255 * sum_v count_v 256^v mod 2^32)
    const uint32_t sE = ((zc_mm + zc_pm) + (zc_mp + zc_pp)) + ((xc_mm + xc_pm) + (xc_mp + xc_pp)) +
                        ((yc_mm + yc_pm) + (yc_mp + yc_pp));
    const uint32_t sF = (fxm + fxp) + (fym + fyp) + (fzm + fzp);
    const uint32_t sV = ((v_mmm + v_pmm) + (v_mpm + v_ppm)) + ((v_mmp + v_pmp) + (v_mpp + v_ppp));
    // x * 0x01010101 = -x / 255 (mod 2^32).  EC change 1 + nE - nF - nV in
    // [-13, 13], area change 6 - 2 nF in [-6, 6], perimeter change 12 - 2 m
    // in [-12, 12]: each byte gets 128 + its change, then loses the 128.
    QuadDelta q;
    q.ec = ((sF + sV - sE) * 0x01010101u + 0x81818181u) ^ 0x80808080u;
    q.area = (sF * 0x02020202u + 0x86868686u) ^ 0x80808080u;
    if (PER) {
        const uint32_t sM =
            ((maj3(fxm, fym, ~ECB(-1, -1, 0)) + maj3(fxp, fym, ~ECB(1, -1, 0))) +
             (maj3(fxm, fyp, ~ECB(-1, 1, 0)) + maj3(fxp, fyp, ~ECB(1, 1, 0)))) +
            ((maj3(fym, fzm, ~ECB(0, -1, -1)) + maj3(fyp, fzm, ~ECB(0, 1, -1))) +
             (maj3(fym, fzp, ~ECB(0, -1, 1)) + maj3(fyp, fzp, ~ECB(0, 1, 1)))) +
            ((maj3(fxm, fzm, ~ECB(-1, 0, -1)) + maj3(fxp, fzm, ~ECB(1, 0, -1))) +
             (maj3(fxm, fzp, ~ECB(-1, 0, 1)) + maj3(fxp, fzp, ~ECB(1, 0, 1))));
        q.per = (sM * 0x02020202u + 0x8C8C8C8Cu) ^ 0x80808080u;
    } else {
        q.per = 0u;
    }
#undef ECB
    return q;
}

// Changes of four horizontally adjacent pixels as signed bytes (byte v =
// pixel v), from the 3 x 3 neighbour level pairs of the pixel pairs (0, 1)
// and (2, 3): n0/n1[(dx+1) + 3*(dy+1)] (index 4 = the pixels themselves).
// Same byte-mask counting as quad_delta.
struct Quad2 {
    uint32_t ec, per;
};

template <bool CONN4>
EC_HD Quad2 quad_delta_2d(const uint32_t (&n0)[9], uint32_t c0, const uint32_t (&n1)[9],
                                               uint32_t c1)
{
    const uint32_t cm0 = c0 | 0x80008000u, cm1 = c1 | 0x80008000u;
    uint32_t b[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const uint32_t k = i > 4 ? 0x00010001u : 0u;
        b[i] = (i == 4) ? 0u : sign_bytes4(cm0 - n0[i] - k, cm1 - n1[i] - k);
    }
    const uint32_t fxm = b[3], fxp = b[5], fym = b[1], fyp = b[7];
    // corner covers: a corner of the pixel is present iff one of its 3 other pixels precedes
    const uint32_t cv_mm = fxm | fym | b[0], cv_pm = fxp | fym | b[2];
    const uint32_t cv_mp = fxm | fyp | b[6], cv_pp = fxp | fyp | b[8];
    const uint32_t sE = (fxm + fxp) + (fym + fyp);
    uint32_t neg = (cv_mm + cv_pm) + (cv_mp + cv_pp);   // digits subtracted from EC
    if (CONN4) {
        // QD corners: a corner becomes QD when only the diagonal precedes and
        // stops being QD when exactly the two edge neighbours precede
        const uint32_t qp = ((b[0] & ~fxm & ~fym) + (b[2] & ~fxp & ~fym)) + ((b[6] & ~fxm & ~fyp) + (b[8] & ~fxp & ~fyp));
        const uint32_t qm = ((fxm & fym & ~b[0]) + (fxp & fym & ~b[2])) + ((fxm & fyp & ~b[6]) + (fxp & fyp & ~b[8]));
        neg = neg + qm - qp;
    }
    // x * 0x01010101 = -x / 255 (mod 2^32).  EC change 1 + nE - nV (+ QD terms)
    // in [-7, 9], perimeter change 4 - 2 nE in [-4, 4]: each byte gets 128 +
    // its change, then loses the 128.
    Quad2 q;
    q.ec = ((neg - sE) * 0x01010101u + 0x81818181u) ^ 0x80808080u;
    q.per = (sE * 0x02020202u + 0x84848484u) ^ 0x80808080u;
    return q;
}

}  // namespace ec
