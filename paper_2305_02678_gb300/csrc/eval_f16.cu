// FP16 tensor-core evaluation: the weight blob (host packing) and the
// FP16 instantiations of the kernel in eval_tc.cuh.
#include "eval_tc.cuh"

namespace nam {

size_t f16_blob_bytes(const Shape& s) {
  if (!f16_supported(s)) return 0;
  return (size_t)f16_lay(s.H, s.frame, s.NH).BYTES;
}

static inline int kmaj(int R, int row, int k) { return (k / 8) * (R * 16) + row * 16 + (k % 8) * 2; }
// the same for 8-bit elements: 8-row x 16-byte core matrices of 16 codes
static inline int kmaj8(int R, int row, int k) { return (k / 16) * (R * 16) + row * 16 + (k % 16); }

static void puth(uint8_t* base, int R, int row, int k, float v) {
  const __half h = __float2half_rn(v);
  std::memcpy(base + kmaj(R, row, k), &h, 2);
}

// v rounded to binary16, stored as FP32 at float index i of base
static void putf(uint8_t* base, int i, float v) {
  const float r = __half2float(__float2half_rn(v));
  std::memcpy(base + 4 * i, &r, 4);
}
static void putf_exact(uint8_t* base, int i, float v) { std::memcpy(base + 4 * i, &v, 4); }

// E4M3 (OCP 8-bit float, "FN" variant: bias 7, no infinities, S.1111.111 the
// only NaN, largest finite 448) of an FP32 value, round to nearest even,
// saturating to +-448.  Written from the format's definition.
static uint8_t e4m3_of(float x) {
  if (std::isnan(x)) return 0x7F;
  const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
  const double a = std::fabs((double)x);
  if (a >= 448.0) return sign | 0x7E;
  if (a < 0.015625) {  // below 2^-6: subnormal codes, spacing 2^-9
    const int m = (int)std::nearbyint(a * 512.0);  // m = 8 is the smallest normal
    return sign | (uint8_t)m;
  }
  int e2;
  const double f = std::frexp(a, &e2);  // a = f 2^e2, f in [0.5, 1)
  int E = e2 - 1;
  int m = (int)std::nearbyint((f * 2.0 - 1.0) * 8.0);
  if (m == 8) {
    m = 0;
    ++E;
  }
  if (E > 8 || (E == 8 && m == 7)) return sign | 0x7E;
  return sign | (uint8_t)(((E + 7) << 3) | m);
}

// The smallest power of two s with amax / s <= 448 (1 for amax = 0): the
// scale under which the largest value maps into the E4M3 range and dividing
// by s is exact.
static double pow2_scale(double amax) {
  double s = 1.0;
  if (amax > 0.0) {
    while (amax / s > 448.0) s *= 2.0;
    while (amax / (s * 0.5) <= 448.0) s *= 0.5;
  }
  return s;
}

// Lay out the FP32 masters, rounded to binary16 (round to nearest even), as
// the kernel's B operands.  frame: form 1 [Wf1 16x8, bf1, Wf2 6x16, bf2],
// form 2 [Wf 12x8, bf]; dec: per layer W [out][in] then b.  FP8: the
// hidden -> hidden layers instead hold E4M3 codes of W / s_w (s_w the
// power-of-two scale of the layer's absmax), twice along K for the (hi, lo)
// input codes, and their FP32 bias; act_scale[l] (the calibrated max |input|
// / 448 of decoder layer l) gives the input scale s_a, the smallest power of
// two >= act_scale[l].  weight_scales_out[l]: s_w of those layers, 0 for the
// others.
int pack_f16_blob(const Shape& s, int precision, const float* frame, const float* dec, const float* act_scale,
                  uint8_t* out, float* weight_scales_out) {
  if (!f16_supported(s)) return -1;
  const bool p8 = precision == NAM_PREC_FP8;
  if (p8 && !act_scale) return -1;
  const int H = s.H, IN = s.in;
  const F16Lay o = f16_lay(H, s.frame, s.NH);
  std::memset(out, 0, (size_t)o.BYTES);
  if (weight_scales_out)
    for (int l = 0; l <= s.NH; ++l) weight_scales_out[l] = 0.0f;
  const float* W1 = dec;  // [H][IN]
  const float* b1 = W1 + H * IN;
  // first MMA: decoder layer 1's z columns, then the frame layer
  for (int n = 0; n < H; ++n)
    for (int k = 0; k < 16; ++k) puth(out + o.B1, o.N1, n, k, W1[n * IN + (k & 7)]);
  if (s.frame == 1) {
    const float* Wf1 = frame;      // [16][8]
    const float* bf1 = Wf1 + 128;  // [16]
    const float* Wf2 = bf1 + 16;   // [6][16]
    const float* bf2 = Wf2 + 96;   // [6]
    for (int j = 0; j < 16; ++j) {
      for (int k = 0; k < 16; ++k) puth(out + o.B1, o.N1, H + j, k, Wf1[j * 8 + (k & 7)]);
      puth(out + o.B1B, 16, j, 0, bf1[j]);
    }
    for (int j = 0; j < 6; ++j) {
      for (int k = 0; k < 32; ++k) puth(out + o.BF2, 16, j, k, Wf2[j * 16 + (k & 15)]);
      putf(out + o.SB, 16 + j, bf2[j]);
    }
  } else if (s.frame == 2) {
    const float* Wf = frame;     // [12][8]
    const float* bf = Wf + 96;   // [12]
    for (int j = 0; j < 12; ++j) {
      for (int k = 0; k < 16; ++k) puth(out + o.B1, o.N1, H + j, k, Wf[j * 8 + (k & 7)]);
      puth(out + o.B1B, 16, j, 0, bf[j]);
    }
  }
  // direction block of layer 1 with its bias
  for (int n = 0; n < H; ++n) {
    for (int k = 0; k < o.ND; ++k) {
      puth(out + o.BD, H, n, k, W1[n * IN + 8 + k]);
      puth(out + o.BD, H, n, o.ND + k, W1[n * IN + 8 + k]);
    }
    puth(out + o.BD, H, n, 2 * o.ND, b1[n]);
  }
  const float* p = b1 + H;
  for (int l = 0; l < s.NH - 1; ++l) {
    const float* Wh = p;
    const float* bh = Wh + H * H;
    uint8_t* dst = out + o.BH + l * H * (H + 16) * 2;
    if (p8) {
      double amax = 0.0;
      for (int i = 0; i < H * H; ++i) amax = std::fmax(amax, std::fabs((double)Wh[i]));
      const double sw = pow2_scale(amax);
      const double sa = pow2_scale((double)act_scale[1 + l] * 448.0);
      for (int n = 0; n < H; ++n) {
        for (int k = 0; k < H; ++k) {
          const uint8_t c = e4m3_of((float)((double)Wh[n * H + k] / sw));
          dst[kmaj8(H, n, k)] = c;
          dst[kmaj8(H, n, H + k)] = c;
        }
        putf(dst + 2 * H * H, n, bh[n]);
      }
      putf_exact(out + o.SB, 2 * l, (float)(1.0 / sa));     // input multiplier 1 / s_a
      putf_exact(out + o.SB, 2 * l + 1, (float)(sa * sw));  // accumulator scale c = s_a s_w
      if (weight_scales_out) weight_scales_out[1 + l] = (float)sw;
    } else {
      for (int n = 0; n < H; ++n) {
        for (int k = 0; k < H; ++k) puth(dst, H, n, k, Wh[n * H + k]);
        puth(dst, H, n, H, bh[n]);
      }
    }
    p = bh + H;
  }
  const float* Wo = p;
  const float* bo = Wo + s.out * H;
  for (int n = 0; n < s.out; ++n) {
    for (int k = 0; k < H; ++k) puth(out + o.BO, 16, n, k, Wo[n * H + k]);
    putf(out + o.SB, 24 + n, bo[n]);
  }
  return 0;
}


size_t tc_blob_bytes(const Shape& s, int precision) {
  if (precision != NAM_PREC_F16 && precision != NAM_PREC_FP8) return 0;
  return f16_blob_bytes(s);
}

int pack_tc_blob(const Shape& s, int precision, const float* frame, const float* dec, const float* act_scale,
                 uint8_t* out, float* weight_scales_out) {
  if (precision != NAM_PREC_F16 && precision != NAM_PREC_FP8) return -1;
  return pack_f16_blob(s, precision, frame, dec, act_scale, out, weight_scales_out);
}

int launch_eval_tc(const LaunchCommon& L, int precision, void* stream) {
  if (precision == NAM_PREC_FP8) return launch_eval_fp8(L, stream);
  return launch_eval_f16(L, stream);
}

int launch_eval_f16(const LaunchCommon& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!f16_supported(L.shape)) return (int)cudaErrorInvalidValue;
  if (L.shape.NH == 3) return f16_frame<64, 3, false>(L, s);
  if (L.shape.H == 16) return f16_frame<16, 2, false>(L, s);
  if (L.shape.H == 32) return f16_frame<32, 2, false>(L, s);
  return f16_frame<64, 2, false>(L, s);
}

}  // namespace nam
