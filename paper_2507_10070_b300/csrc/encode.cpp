// Compressed navigation vectors: float32 -> BF16 and float32 -> FP8-E4M3
// (host-side encoders used when an index is loaded with compressed
// navigation; the device decodes with CUDA's own conversions).
//
// BF16: the upper 16 bits of the float32, rounded to nearest, ties to even.
// FP8-E4M3 (OCP 8-bit floating point, E4M3 variant): sign, 4 exponent bits
// (bias 7), 3 mantissa bits; largest finite magnitude 448 (S.1111.110); no
// infinities; S.1111.111 is NaN.  Encoding rounds to nearest, ties to even,
// and saturates finite values beyond 448 to +-448; subnormals have exponent
// field 0 and value m * 2^-9.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/ann.h"

namespace {

uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return static_cast<uint16_t>((u >> 16) | 0x40);  // NaN stays NaN
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return static_cast<uint16_t>(u >> 16);
}

uint8_t to_e4m3(float f) {
  if (std::isnan(f)) return 0x7f;
  const uint8_t sign = std::signbit(f) ? 0x80 : 0x00;
  double a = std::fabs(static_cast<double>(f));
  if (a >= 448.0) return sign | 0x7e;  // saturate
  if (a < std::ldexp(1.0, -10)) return sign;  // below half the smallest subnormal (2^-9): +-0
  int e;
  const double m = std::frexp(a, &e);  // a = m * 2^e, m in [0.5, 1)
  int exp_field = e - 1 + 7;           // value = 1.f * 2^(e-1)
  if (exp_field >= 1) {
    // normal: 3 mantissa bits
    double scaled = std::ldexp(a, 3 - (e - 1));  // in [8, 16)
    double r = std::nearbyint(scaled);           // ties to even (default rounding mode)
    if (r == 16.0) {
      r = 8.0;
      ++exp_field;
    }
    if (exp_field > 15 || (exp_field == 15 && r - 8.0 > 6.0)) return sign | 0x7e;
    return sign | static_cast<uint8_t>(exp_field << 3) | static_cast<uint8_t>(static_cast<int>(r) - 8);
  }
  // subnormal: value = mant * 2^-9, mant in 0..7
  const double r = std::nearbyint(std::ldexp(a, 9));
  if (r >= 8.0) return sign | 0x08;  // rounds up to the smallest normal
  return sign | static_cast<uint8_t>(r);
  (void)m;
}

}  // namespace

extern "C" int ann_encode_bf16(const float* x, int64_t n, uint16_t* out) {
  if ((!x || !out) && n > 0) return ANN_EINVAL;
  for (int64_t i = 0; i < n; ++i) out[i] = to_bf16(x[i]);
  return ANN_OK;
}

extern "C" int ann_encode_fp8e4m3(const float* x, int64_t n, float scale, uint8_t* out) {
  if (((!x || !out) && n > 0) || !(scale > 0.f)) return ANN_EINVAL;
  for (int64_t i = 0; i < n; ++i) out[i] = to_e4m3(x[i] * scale);
  return ANN_OK;
}
