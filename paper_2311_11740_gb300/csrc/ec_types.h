// ec_types.h -- the vertex types of Tables 1 and 2 as mask -> type tables.
#pragma once
#include <stdint.h>

namespace ec {

// ------------------------------------------------------------ vertex types
//
// The types of Tables 1 and 2 are the classes of neighbourhood patterns under
// the symmetries of the square (8) and the cube (48).  Each table row draws
// one pattern; those drawings, written as masks (bit x + 2y (+ 4z); for the
// cube pictures the macro's eight node positions are (0,1,1) (1,1,1) (0,1,0)
// (1,1,0) (0,0,1) (1,0,1) (0,0,0) (1,0,0) in (x, y, z)), are the rows'
// representatives below, in the tables' row order.  A mask's type is the row
// whose representative lies in the mask's class.  Type 0 is the empty
// neighbourhood; 2D: Q0, Q1, Q2, QD, Q3, Q4.
constexpr int kTypes2 = 6, kTypes3 = 22;
constexpr uint8_t kTable1Reps[kTypes2] = {0x0, 0x4, 0x5, 0x6, 0x7, 0xF};
constexpr uint8_t kTable2Reps[kTypes3] = {0x00, 0x40, 0xC0, 0x48, 0x42, 0xC4, 0xC1, 0x49, 0xCC, 0xD4, 0xE4,
                                          0xC6, 0x66, 0x69, 0x57, 0x67, 0x79, 0x77, 0x7B, 0xE7, 0xFD, 0xFF};

struct TypeTable2D { uint8_t t[16]; };
struct TypeTable3D { uint8_t t[256]; };

// Image of mask m under the symmetry (axis permutation number p, reflection
// bits f) of the n-cube, n = 2 or 3: the cell at c goes to c' with
// c'[a] = c[perm[a]] ^ f_a.
constexpr unsigned sym_image(unsigned m, int n, int p, unsigned f)
{
    int perm[3] = {0, 1, 2};
    // the six permutations of three axes (the first two for n = 2)
    constexpr int P3[6][3] = {{0, 1, 2}, {1, 0, 2}, {0, 2, 1}, {2, 1, 0}, {1, 2, 0}, {2, 0, 1}};
    for (int a = 0; a < 3; a++) perm[a] = P3[p][a];
    unsigned out = 0;
    for (unsigned b = 0; b < (1u << n); b++) {
        if (!(m >> b & 1u)) continue;
        unsigned nb = 0;
        for (int a = 0; a < n; a++) nb |= (((b >> perm[a]) & 1u) ^ ((f >> a) & 1u)) << a;
        out |= 1u << nb;
    }
    return out;
}

// Smallest mask of m's class.
constexpr unsigned class_min(unsigned m, int n)
{
    unsigned best = m;
    const int np = n == 2 ? 2 : 6;
    for (int p = 0; p < np; p++)
        for (unsigned f = 0; f < (1u << n); f++) {
            const unsigned im = sym_image(m, n, p, f);
            if (im < best) best = im;
        }
    return best;
}

constexpr TypeTable3D make_type_table_3d()
{
    TypeTable3D t{};
    unsigned rep[kTypes3] = {};
    for (int r = 0; r < kTypes3; r++) rep[r] = class_min(kTable2Reps[r], 3);
    for (unsigned m = 0; m < 256; m++) {
        const unsigned c = class_min(m, 3);
        t.t[m] = 0xFF;   // no row: caught by ec_selfcheck_rules
        for (int r = 0; r < kTypes3; r++)
            if (rep[r] == c) t.t[m] = (uint8_t)r;
    }
    return t;
}

constexpr TypeTable2D make_type_table_2d()
{
    TypeTable2D t{};
    unsigned rep[kTypes2] = {};
    for (int r = 0; r < kTypes2; r++) rep[r] = class_min(kTable1Reps[r], 2);
    for (unsigned m = 0; m < 16; m++) {
        const unsigned c = class_min(m, 2);
        t.t[m] = 0xFF;
        for (int r = 0; r < kTypes2; r++)
            if (rep[r] == c) t.t[m] = (uint8_t)r;
    }
    return t;
}

}  // namespace ec
