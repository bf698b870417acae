// ec_swar.h -- per-voxel contribution changes for two voxels at once.
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
// The contribution change then follows from which faces, edges and vertices
// of c's closure are already present (see voxel_delta_3d in ec_rules.h):
//   edge covers   (12): an edge of c is present iff one of its 3 other voxels precedes
//   corner covers  (8): a vertex of c is present iff one of its 7 other voxels precedes
//   face bits      (6): a face of c is present iff the voxel across it precedes
//   crease minus  (12): the edge weight drops iff more face neighbours than
//                       diagonal neighbours around it precede (majority of a1, a2, not d)
// computed bitwise on the comparison words (both lanes at once), gathered
// into per-voxel bit sets with `prmt` sign replication (each sign bit of a
// comparison word becomes a byte mask), and counted with popc.
#pragma once
#include <stdint.h>

#include "ec_rules.h"

namespace ec {

// prmt.b32 in its default mode with all four selector nibbles asking for
// sign replication: output bytes = msb of (a.byte1, b.byte1, a.byte3, b.byte3)
// replicated over 8 bits, i.e. the lane-0 and lane-1 comparison bits of a and b.
EC_HD uint32_t sign_bytes(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(0xFBD9u));
    return d;
#else
    const uint32_t m0 = (a >> 15) & 1u ? 0xFFu : 0u;
    const uint32_t m1 = (b >> 15) & 1u ? 0xFFu : 0u;
    const uint32_t m2 = (a >> 31) & 1u ? 0xFFu : 0u;
    const uint32_t m3 = (b >> 31) & 1u ? 0xFFu : 0u;
    return m0 | (m1 << 8) | (m2 << 16) | (m3 << 24);
#endif
}

// Add the comparison bits of words a and b to a per-voxel bit set: voxel 0
// gets them at bits pa and 8+pb, voxel 1 at 16+pa and 24+pb.
template <int PA, int PB>
EC_HD uint32_t gather2(uint32_t acc, uint32_t a, uint32_t b)
{
    constexpr uint32_t K = (1u << PA) | (1u << (8 + PB)) | (1u << (16 + PA)) | (1u << (24 + PB));
    return acc | (sign_bytes(a, b) & K);
}

EC_HD uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (a & c) | (b & c); }

// Largest level count of the 3D paths that use pair_delta: every key,
// including the never-active level L, fits a 16-bit lane below 0x8000.
constexpr int kMaxFastL3 = 32767;

struct PairDelta {
    int ec[2], per[2], area[2];
};

// n[(dx+1) + 3*(dy+1) + 9*(dz+1)]: neighbour key pairs (both voxels shifted
// by the same offset); c: the two centre keys.
template <bool PER>
EC_HD PairDelta pair_delta(const uint32_t (&n)[27], uint32_t c)
{
    const uint32_t cm = c | 0x80008000u;
    uint32_t d[27];
#pragma unroll
    for (int i = 0; i < 27; i++) d[i] = (i == 13) ? 0u : cm - n[i] - (i > 13 ? 0x00010001u : 0u);
#define ECD(dx, dy, dz) d[((dx) + 1) + 3 * ((dy) + 1) + 9 * ((dz) + 1)]
    const uint32_t fxm = ECD(-1, 0, 0), fxp = ECD(1, 0, 0);
    const uint32_t fym = ECD(0, -1, 0), fyp = ECD(0, 1, 0);
    const uint32_t fzm = ECD(0, 0, -1), fzp = ECD(0, 0, 1);
    // edge covers, named by the signs of the two offsets that are non-zero
    const uint32_t zc_mm = fxm | fym | ECD(-1, -1, 0), zc_pm = fxp | fym | ECD(1, -1, 0);
    const uint32_t zc_mp = fxm | fyp | ECD(-1, 1, 0), zc_pp = fxp | fyp | ECD(1, 1, 0);
    const uint32_t xc_mm = fym | fzm | ECD(0, -1, -1), xc_pm = fyp | fzm | ECD(0, 1, -1);
    const uint32_t xc_mp = fym | fzp | ECD(0, -1, 1), xc_pp = fyp | fzp | ECD(0, 1, 1);
    const uint32_t yc_mm = fxm | fzm | ECD(-1, 0, -1), yc_pm = fxp | fzm | ECD(1, 0, -1);
    const uint32_t yc_mp = fxm | fzp | ECD(-1, 0, 1), yc_pp = fxp | fzp | ECD(1, 0, 1);
    // corner covers: the vertex (sx, sy, sz) of c
#define VC(sx, sy, sz, zc, xc, yc) ((zc) | (xc) | (yc) | ECD(sx, sy, sz))
    const uint32_t v_mmm = VC(-1, -1, -1, zc_mm, xc_mm, yc_mm), v_pmm = VC(1, -1, -1, zc_pm, xc_mm, yc_pm);
    const uint32_t v_mpm = VC(-1, 1, -1, zc_mp, xc_pm, yc_mm), v_ppm = VC(1, 1, -1, zc_pp, xc_pm, yc_pm);
    const uint32_t v_mmp = VC(-1, -1, 1, zc_mm, xc_mp, yc_mp), v_pmp = VC(1, -1, 1, zc_pm, xc_mp, yc_pp);
    const uint32_t v_mpp = VC(-1, 1, 1, zc_mp, xc_pp, yc_mp), v_ppp = VC(1, 1, 1, zc_pp, xc_pp, yc_pp);
#undef VC
    // two independent chains per bit set keep the dependent LOP3s short
    uint32_t pos_a = 0, pos_b = 0, neg_a = 0, neg_b = 0;
    pos_a = gather2<0, 0>(pos_a, zc_mm, zc_pm);
    pos_b = gather2<1, 1>(pos_b, zc_mp, zc_pp);
    pos_a = gather2<2, 2>(pos_a, xc_mm, xc_pm);
    pos_b = gather2<3, 3>(pos_b, xc_mp, xc_pp);
    pos_a = gather2<4, 4>(pos_a, yc_mm, yc_pm);
    pos_b = gather2<5, 5>(pos_b, yc_mp, yc_pp);
    neg_a = gather2<0, 0>(neg_a, fxm, fxp);
    neg_b = gather2<1, 1>(neg_b, fym, fyp);
    neg_a = gather2<2, 2>(neg_a, fzm, fzp);
    neg_b = gather2<3, 3>(neg_b, v_mmm, v_pmm);
    neg_a = gather2<4, 4>(neg_a, v_mpm, v_ppm);
    neg_b = gather2<5, 5>(neg_b, v_mmp, v_pmp);
    neg_a = gather2<6, 6>(neg_a, v_mpp, v_ppp);
    const uint32_t pos = pos_a | pos_b, neg = neg_a | neg_b;
    PairDelta r;
    const int pos0 = popc32(pos & 0xFFFFu), pos1 = popc32(pos >> 16);
    const int neg0 = popc32(neg & 0xFFFFu), neg1 = popc32(neg >> 16);
    const int f0 = popc32(neg & 0x0707u), f1 = popc32(neg & 0x07070000u);
    r.ec[0] = 1 + pos0 - neg0;
    r.ec[1] = 1 + pos1 - neg1;
    r.area[0] = 6 - 2 * f0;
    r.area[1] = 6 - 2 * f1;
    if (PER) {
        uint32_t mi_a = 0, mi_b = 0;
        mi_a = gather2<0, 0>(mi_a, maj3(fxm, fym, ~ECD(-1, -1, 0)), maj3(fxp, fym, ~ECD(1, -1, 0)));
        mi_b = gather2<1, 1>(mi_b, maj3(fxm, fyp, ~ECD(-1, 1, 0)), maj3(fxp, fyp, ~ECD(1, 1, 0)));
        mi_a = gather2<2, 2>(mi_a, maj3(fym, fzm, ~ECD(0, -1, -1)), maj3(fyp, fzm, ~ECD(0, 1, -1)));
        mi_b = gather2<3, 3>(mi_b, maj3(fym, fzp, ~ECD(0, -1, 1)), maj3(fyp, fzp, ~ECD(0, 1, 1)));
        mi_a = gather2<4, 4>(mi_a, maj3(fxm, fzm, ~ECD(-1, 0, -1)), maj3(fxp, fzm, ~ECD(1, 0, -1)));
        mi_b = gather2<5, 5>(mi_b, maj3(fxm, fzp, ~ECD(-1, 0, 1)), maj3(fxp, fzp, ~ECD(1, 0, 1)));
        const uint32_t mi = mi_a | mi_b;
        r.per[0] = 12 - 2 * popc32(mi & 0xFFFFu);
        r.per[1] = 12 - 2 * popc32(mi >> 16);
    } else {
        r.per[0] = r.per[1] = 0;
    }
#undef ECD
    return r;
}

}  // namespace ec
