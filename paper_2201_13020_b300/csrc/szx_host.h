// szx_host.h -- host-side argument helpers shared by the C ABI's files (not
// part of the ABI).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "szx.h"

namespace szx {

// b: a power of two in [32, 1024].
inline bool block_ok(uint32_t b) { return b >= 32 && b <= 1024 && (b & (b - 1)) == 0; }

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// The bound actually used, as the bit pattern of the value's type: for f64
// the double itself; for f32 the largest float <= eb (rounding toward zero).
inline uint64_t bound_bits(double eb, szx_dtype d) {
    if (d == SZX_F64) {
        uint64_t u;
        std::memcpy(&u, &eb, 8);
        return u;
    }
    float f = static_cast<float>(eb);
    if (static_cast<double>(f) > eb) f = std::nextafterf(f, 0.0f);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

}  // namespace szx
