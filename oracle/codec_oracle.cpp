// FP64/integer CPU oracle of the cluster codec: the conversion of cluster
// properties from the reconstruction's floating-point format to integers with
// as many bits as the detector resolution needs (Sec. 4, step 2).
//
// Test infrastructure only: tests, smoke() and the CPU baseline of the
// benchmark use it; the library never does.  It shares no code with the CUDA
// path.
//
// What the paper fixes (Sec. 4, step 2): cluster size and charge are stored
// with a precision relative to their own magnitude -- in the integer
// representation every bit lying more than n places after the first non-zero
// bit becomes zero, with rounding, n = 3 for the size and n = 4 for the charge.
//
// Readings (the paper gives neither units nor field widths):
//  - positions y, z: fixed point with a step of 2^-6 cm, rounded to nearest
//    (ties to even); y in int16, z in int32 (continuous read-out z reaches
//    metres); saturated to the field's range;
//  - pad row: uint8;
//  - charges q_tot, q_max: integer ADC counts (rounded to nearest, ties to
//    even, negative -> 0), saturated to uint16, then dynamic precision n = 4;
//  - sizes sigma_y, sigma_z: fixed point with a step of 2^-7 cm in uint8, then
//    dynamic precision n = 3;
//  - "proper rounding" of the dynamic precision = to the nearest value that
//    keeps n bits after the leading one, ties upward; a result above the field
//    maximum becomes the largest such value that fits;
//  - a non-finite value or a row outside [0, n_rows) marks the cluster bad
//    (counted); its codes still follow the rules above with NaN -> 0.
#include <cmath>
#include <cstdint>

namespace {

// Nearest integer, ties to even, of an exactly representable double.
double round_even(double v) { return std::nearbyint(v); }  // default FE_TONEAREST

int64_t to_fixed(double v, double scale, int64_t lo, int64_t hi) {
  if (std::isnan(v)) return 0;
  const double s = round_even(v * scale);  // v * 2^k is exact in binary64
  if (s <= (double)lo) return lo;
  if (s >= (double)hi) return hi;
  return (int64_t)s;
}

}  // namespace

extern "C" {

// Dynamic precision (Sec. 4, step 2): keep the leading one of v and the n bits
// after it; round the rest away (half upward); clamp into `width` bits.
uint32_t orc_dyn_round(uint32_t v, int n, int width) {
  if (v == 0) return 0;
  int lead = 0;  // index of the first non-zero bit
  for (int b = 0; b < 32; ++b)
    if ((v >> b) & 1u) lead = b;
  const int drop = lead - n;  // bits to clear below the kept ones
  uint64_t r = v;
  if (drop > 0) {
    const uint64_t unit = 1ull << drop;
    r = ((r + unit / 2) / unit) * unit;
  }
  const uint64_t field_max = (1ull << width) - 1;
  if (r > field_max) {  // the largest value with n bits after its leading one
    r = ((1ull << (n + 1)) - 1) << (width - n - 1);
  }
  return (uint32_t)r;
}

// Encodes n clusters.  Returns the number of bad clusters.
int64_t orc_encode_clusters(int64_t n, int n_rows, const float* y, const float* z, const int32_t* row,
                            const float* q_tot, const float* q_max, const float* sigma_y, const float* sigma_z,
                            int16_t* cy, int32_t* cz, uint8_t* crow, uint16_t* cqt, uint16_t* cqm, uint8_t* csy,
                            uint8_t* csz) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double v[6] = {y[i], z[i], q_tot[i], q_max[i], sigma_y[i], sigma_z[i]};
    bool ok = row[i] >= 0 && row[i] < n_rows;
    for (double e : v) ok = ok && std::isfinite(e);
    if (!ok) ++bad;
    cy[i] = (int16_t)to_fixed(v[0], 64.0, INT16_MIN, INT16_MAX);
    cz[i] = (int32_t)to_fixed(v[1], 64.0, INT32_MIN, INT32_MAX);
    crow[i] = (row[i] >= 0 && row[i] < n_rows) ? (uint8_t)row[i] : 0;
    cqt[i] = (uint16_t)orc_dyn_round((uint32_t)to_fixed(v[2], 1.0, 0, 65535), 4, 16);
    cqm[i] = (uint16_t)orc_dyn_round((uint32_t)to_fixed(v[3], 1.0, 0, 65535), 4, 16);
    csy[i] = (uint8_t)orc_dyn_round((uint32_t)to_fixed(v[4], 128.0, 0, 255), 3, 8);
    csz[i] = (uint8_t)orc_dyn_round((uint32_t)to_fixed(v[5], 128.0, 0, 255), 3, 8);
  }
  return bad;
}

}  // extern "C"
