// One-level straight-line programs of the 2x2 recursions, on words of bits
// (every bit position is an independent instance). Written for the GPU path
// from the paper's equations; host code uses the same functions to read off
// the 0/1 matrices the scheduler needs for its depth-first levels.
//
// Block order: index 2*r + c for block (r, c), i.e. (X00, X01, X10, X11);
// products h = 0..6 as in the paper.
#pragma once

#include <stdint.h>

namespace bmm {
namespace slp {

// Forward basis change, in place: phi for A, psi for B (phi = psi in both
// alternative-basis variants; identity for Strassen–Winograd).
template <int V, typename W>
__host__ __device__ __forceinline__ void phi(W* x) {
    if (V == 1) {  // Eq. mb-fwdbasisrecurrence
        x[3] = x[1] ^ x[2] ^ x[3];
    } else if (V == 2) {  // Eq. ab-fwdbasisrecurrence
        x[3] = x[1] ^ x[3];
        x[2] = x[3] ^ x[2];
    }
}

// Inverse basis change chi, in place.
template <int V, typename W>
__host__ __device__ __forceinline__ void chi(W* x) {
    if (V == 1) {  // Eq. mb-revbasisrecurrence
        x[1] = x[1] ^ x[3];
        x[2] = x[2] ^ x[3];
    } else if (V == 2) {  // Eq. ab-revbasisrecurrence (X10 uses the old X11)
        x[2] = x[2] ^ x[3];
        x[3] = x[1] ^ x[3];
    }
}

// Left-operand combinations T_h (alpha; xi for Strassen–Winograd).
template <int V, typename W>
__host__ __device__ __forceinline__ void alpha(const W* a, W* t) {
    if (V == 0) {  // Eq. sw-input
        t[0] = a[2] ^ a[3];
        t[1] = a[1];
        t[2] = a[1] ^ a[3];
        t[3] = a[2] ^ t[2];
        t[4] = a[0] ^ t[3];
        t[5] = a[2];
        t[6] = a[0];
    } else if (V == 1) {  // Eq. mb-tsrecurrence
        t[0] = a[0];
        t[1] = a[1];
        t[2] = a[2];
        t[3] = a[3];
        t[4] = a[0] ^ a[3];
        t[5] = a[1] ^ a[3];
        t[6] = a[2] ^ a[3];
    } else {  // Eq. ab-tsrecurrence
        t[0] = a[0];
        t[1] = a[1];
        t[2] = a[2];
        t[3] = a[3];
        t[4] = a[0] ^ a[2];
        t[5] = a[1] ^ a[2];
        t[6] = a[2] ^ a[3];
    }
}

// Right-operand combinations S_h (beta; eta for Strassen–Winograd). b holds
// the blocks of B (not of its transpose) in (B00, B01, B10, B11) order.
template <int V, typename W>
__host__ __device__ __forceinline__ void beta(const W* b, W* s) {
    if (V == 0) {  // Eq. sw-input
        s[0] = b[2] ^ b[3];
        s[1] = b[2];
        s[2] = b[1] ^ b[3];
        s[3] = b[2] ^ s[2];
        s[4] = b[1];
        s[5] = b[0] ^ s[3];
        s[6] = b[0];
    } else if (V == 1) {  // Eq. mb-tsrecurrence
        s[0] = b[0];
        s[1] = b[2];
        s[2] = b[0] ^ b[3];
        s[3] = b[3];
        s[4] = b[1];
        s[5] = b[1] ^ b[3];
        s[6] = b[2] ^ b[3];
    } else {  // Eq. ab-tsrecurrence
        s[0] = b[0];
        s[1] = b[2] ^ b[3];
        s[2] = b[2];
        s[3] = b[3];
        s[4] = b[1];
        s[5] = b[1] ^ b[2];
        s[6] = b[0] ^ b[2];
    }
}

// Output combinations: C-blocks from the seven products (gamma; zeta for
// Strassen–Winograd).
template <int V, typename W>
__host__ __device__ __forceinline__ void gamma(const W* q, W* c) {
    if (V == 0) {  // Eq. sw-output
        const W u0 = q[1] ^ q[3];
        const W u1 = q[2] ^ u0;
        const W u2 = q[4] ^ u0;
        c[0] = q[1] ^ q[6];
        c[1] = q[0] ^ u2;
        c[2] = q[5] ^ u1;
        c[3] = q[0] ^ u1;
    } else if (V == 1) {  // Eq. mb-qrecurrence
        c[0] = q[0] ^ q[1];
        c[1] = q[4] ^ q[6];
        c[2] = q[2] ^ q[5];
        c[3] = q[1] ^ q[3] ^ q[5] ^ q[6];
    } else {  // Eq. ab-qrecurrence
        const W r = q[1] ^ q[2] ^ q[4];
        c[0] = q[0] ^ q[1];
        c[1] = r ^ q[5];
        c[2] = r ^ q[6];
        c[3] = q[3] ^ q[4];
    }
}

// Combined standard-basis operators of one level: xi = alpha phi,
// eta = beta psi, zeta = chi gamma, as 0/1 masks read off the programs above
// (xi_mask[h] bit q: block q of A enters T_h; zeta_mask[q] bit h: product h
// enters block q of C).
template <int V>
inline void level_masks(uint32_t xi_mask[7], uint32_t eta_mask[7], uint32_t zeta_mask[4]) {
    for (int h = 0; h < 7; h++) xi_mask[h] = eta_mask[h] = 0;
    for (int q = 0; q < 4; q++) {
        uint32_t x[4] = {0, 0, 0, 0}, t[7];
        x[q] = 1;
        phi<V>(x);
        alpha<V>(x, t);
        for (int h = 0; h < 7; h++) xi_mask[h] |= (t[h] & 1u) << q;
        uint32_t y[4] = {0, 0, 0, 0}, s[7];
        y[q] = 1;
        phi<V>(y);
        beta<V>(y, s);
        for (int h = 0; h < 7; h++) eta_mask[h] |= (s[h] & 1u) << q;
    }
    for (int q = 0; q < 4; q++) zeta_mask[q] = 0;
    for (int h = 0; h < 7; h++) {
        uint32_t qv[7] = {0, 0, 0, 0, 0, 0, 0}, c[4];
        qv[h] = 1;
        gamma<V>(qv, c);
        chi<V>(c);
        for (int q = 0; q < 4; q++) zeta_mask[q] |= (c[q] & 1u) << h;
    }
}

}  // namespace slp
}  // namespace bmm
