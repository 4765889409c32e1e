// Sharded evaluation: contiguous shard ranges and the rank-ordered combine of
// the shards' compensated partial sums (host only; no CUDA call).
#include <cmath>
#include <cstdint>

#include "api_internal.h"

namespace {

struct HPair {
  double s, c;
};

// Exact two-sum merge of compensated pairs (the same merge as the device
// reduction tree's).
HPair merge(HPair a, HPair b) {
  const double s = a.s + b.s;
  const double bb = s - a.s;
  const double e = (a.s - (s - bb)) + (b.s - bb);
  return {s, (a.c + b.c) + e};
}

constexpr int32_t kThetaBadBit = 1 << 30;

}  // namespace

using namespace rf;

extern "C" rf_status rf_shard(int64_t n, int64_t align, int32_t rank, int32_t world, int64_t* lo, int64_t* hi) {
  if (n < 0 || align < 1 || world < 1 || rank < 0 || rank >= world || !lo || !hi) {
    set_error("rf_shard: bad argument");
    return RF_E_INVALID;
  }
  const int64_t C = (n + align - 1) / align;
  // floor(r C / world) without overflow for any realistic C (C < 2^62 / world)
  const int64_t u0 = (int64_t)(((__int128)C * rank) / world);
  const int64_t u1 = (int64_t)(((__int128)C * (rank + 1)) / world);
  *lo = u0 * align < n ? u0 * align : n;
  *hi = rank + 1 == world ? n : (u1 * align < n ? u1 * align : n);
  return RF_OK;
}

extern "C" rf_status rf_combine_partials(const double* pairs, const int32_t* flags, int32_t world, int32_t n_sets,
                                         int32_t n_free, double* out, int32_t* flags_out) {
  if (!pairs || !flags || !out || !flags_out || world < 1 || n_sets < 0 || n_free < 0) {
    set_error("rf_combine_partials: bad argument");
    return RF_E_INVALID;
  }
  const int Q = 1 + n_free;
  bool any = false;
  for (int32_t s = 0; s < n_sets; ++s) {
    int64_t bad = 0;
    bool dom = false;
    for (int32_t r = 0; r < world; ++r) {
      const int32_t f = flags[(int64_t)r * n_sets + s];
      dom = dom || (f & kThetaBadBit) != 0;
      bad += f & (kThetaBadBit - 1);
    }
    const int32_t f = (int32_t)(bad < kThetaBadBit - 1 ? bad : kThetaBadBit - 1) | (dom ? kThetaBadBit : 0);
    flags_out[s] = f;
    any = any || f != 0;
    for (int q = 0; q < Q; ++q) {
      HPair acc{0.0, 0.0};
      for (int32_t r = 0; r < world; ++r) {
        const double* p = pairs + (((int64_t)r * n_sets + s) * Q + q) * 2;
        acc = r == 0 ? HPair{p[0], p[1]} : merge(acc, {p[0], p[1]});
      }
      const double v = -(acc.s + acc.c);
      out[(int64_t)s * Q + q] = (q == 0 && f != 0) ? INFINITY : v;
    }
  }
  if (any) {
    set_error("pdf <= 0 or not finite for some event, or parameters outside a pdf's domain");
    return RF_E_DOMAIN;
  }
  return RF_OK;
}
