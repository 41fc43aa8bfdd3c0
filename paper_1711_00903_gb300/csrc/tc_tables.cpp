// Host side of the tensor-core BP3.0 operator: the per-degree table of B
// fragments (tc_layout.h) built from the FP64 basis.
#include <cmath>
#include <cstdint>

#include "fem_internal.h"
#include "tc_layout.h"

namespace fem {
namespace {

// IEEE binary16 encoding of x, rounded to nearest (ties to even), with
// subnormals; |x| beyond the largest finite value encodes infinity.
uint16_t to_f16(double x) {
    const uint16_t sign = std::signbit(x) ? 0x8000u : 0u;
    double a = std::fabs(x);
    if (a == 0.0) return sign;
    if (std::isnan(x)) return 0x7e00u;
    int e;
    std::frexp(a, &e);  // a = f 2^e, f in [0.5, 1): leading bit at 2^(e-1)
    int E = e - 1;
    if (E < -14) {  // subnormal: multiples of 2^-24
        const double k = std::nearbyint(std::ldexp(a, 24));
        return (uint16_t)(sign | (uint16_t)k);  // k = 1024 is the smallest normal, same bits
    }
    double k = std::nearbyint(std::ldexp(a, 10 - E));  // in [1024, 2048]
    if (k >= 2048.0) {
        k = 1024.0;
        E += 1;
    }
    if (E > 15) return (uint16_t)(sign | 0x7c00u);
    return (uint16_t)(sign | (uint16_t)((E + 15) << 10) | (uint16_t)(k - 1024.0));
}

double from_f16(uint16_t h) {
    const int E = (h >> 10) & 0x1f, M = h & 0x3ff;
    const double s = (h & 0x8000u) ? -1.0 : 1.0;
    if (E == 0) return s * std::ldexp((double)M, -24);
    if (E == 31) return M ? NAN : s * INFINITY;
    return s * std::ldexp(1024.0 + M, E - 25);
}

// Entry Op[o][k] of the 1D operator of a table slot.
double op_entry(const HostBasis &h, int op, int o, int k) {
    switch (op) {
        case TC_I: return h.I[o * h.n + k];    // interpolation (m x n)
        case TC_DT: return h.Dt[o * h.m + k];  // Gauss-point derivative (m x m)
        case TC_DTT: return h.Dt[k * h.m + o]; // its transpose
        case TC_IT: return h.I[k * h.n + o];   // projection I^T (n x m)
        case TC_D: return h.D[o * h.n + k];    // GLL derivative (n x n)
        default: return h.D[k * h.n + o];      // its transpose
    }
}

// Value of the B operand at position p of the K axis and output column o.
uint16_t b_value(const HostBasis &h, int op, int p, int o) {
    const int P = tc_P(h.N, op), Q = tc_Q(h.N, op);
    const int raw = tc_raw(Q, p);
    if (o >= P || raw < 0) return 0;
    const double x = op_entry(h, op, o, raw);
    const uint16_t hi = to_f16(x);
    switch (tc_seg(Q, p)) {
        case 0: return hi;
        case 1: return to_f16(std::ldexp(from_f16(hi), -11));
        default: return to_f16(x - from_f16(hi));
    }
}

}  // namespace

int64_t tc_table_words(int N) { return (int64_t)tc_total_tiles(N) * 32 * 2; }

// words: tc_table_words(N) 32-bit words; per tile, per lane (g = lane / 4,
// t = lane % 4): b0 = {B[16ks + 2t][8nt + g], B[16ks + 2t + 1][...]},
// b1 = {B[16ks + 8 + 2t][...], B[16ks + 9 + 2t][...]}, first element in
// the low half.
void build_tc_table(const HostBasis &h, uint32_t *words) {
    for (int op = 0; op < TC_OPS; op++) {
        const int P = tc_P(h.N, op), Q = tc_Q(h.N, op), NT = tc_nt(P), KS = tc_ks(Q);
        uint32_t *base = words + (int64_t)tc_offset(h.N, op) * 64;
        for (int nt = 0; nt < NT; nt++)
            for (int ks = 0; ks < KS; ks++)
                for (int lane = 0; lane < 32; lane++) {
                    const int g = lane >> 2, t = lane & 3, o = 8 * nt + g;
                    uint32_t *w = base + ((int64_t)(nt * KS + ks) * 32 + lane) * 2;
                    for (int half = 0; half < 2; half++) {
                        const int p = 16 * ks + 8 * half + 2 * t;
                        w[half] = (uint32_t)b_value(h, op, p, o) | ((uint32_t)b_value(h, op, p + 1, o) << 16);
                    }
                }
    }
}

}  // namespace fem
