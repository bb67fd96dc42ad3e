// pp_convert.cuh -- field value conversion on the device (Sec. 3.3).
//
// Each function reads one field's data bytes and returns kConvOk with the
// value's bit pattern, kConvEmpty for an empty field, or kConvFail.  The
// accepted syntax is stated in parparaw.h next to pp_type.
#pragma once
#include <cstdint>

#include "pp_types.h"

namespace pp {

constexpr int kConvOk = 0, kConvEmpty = 1, kConvFail = 2;
constexpr int kNumericMaxLen = 64;

// 10^k, k <= 22: every one is an exactly representable double.
static __device__ __constant__ double kPow10[23] = {1e0,  1e1,  1e2,  1e3,  1e4,  1e5,  1e6,  1e7,
                                             1e8,  1e9,  1e10, 1e11, 1e12, 1e13, 1e14, 1e15,
                                             1e16, 1e17, 1e18, 1e19, 1e20, 1e21, 1e22};
// days before month m (0-based) in a common year
static __device__ __constant__ int kDaysBefore[12] = {0, 31, 59, 90, 120, 151, 181, 212, 243, 273, 304, 334};
static __device__ __constant__ int kDaysIn[12] = {31, 28, 31, 30, 31, 30, 31, 31, 30, 31, 30, 31};
// "Jan".."Dec" packed little-endian into 24 bits
static __device__ __constant__ uint32_t kMonthNames[12] = {
    0x6E614Au, 0x626546u, 0x72614Du, 0x727041u, 0x79614Du, 0x6E754Au,
    0x6C754Au, 0x677541u, 0x706553u, 0x74634Fu, 0x766F4Eu, 0x636544u};

__device__ __forceinline__ bool is_leap(int y) {
  return (y % 4 == 0) && ((y % 100 != 0) || (y % 400 == 0));
}

// Days from 1970-01-01 to y-m-d (proleptic Gregorian): whole years before y
// counted from 0001-01-01 with the 4/100/400 leap rule, then whole months,
// then days, minus the 719162 days from 0001-01-01 to 1970-01-01.
__device__ __forceinline__ int64_t days_since_epoch(int y, int m, int d) {
  const int64_t y1 = y - 1;
  const int64_t years = 365 * y1 + y1 / 4 - y1 / 100 + y1 / 400;
  const int64_t months = kDaysBefore[m - 1] + ((m > 2 && is_leap(y)) ? 1 : 0);
  return years + months + (d - 1) - 719162;
}

__device__ __forceinline__ bool valid_date(int y, int m, int d) {
  if (y < 1 || m < 1 || m > 12 || d < 1) return false;
  const int dim = kDaysIn[m - 1] + ((m == 2 && is_leap(y)) ? 1 : 0);
  return d <= dim;
}

__device__ __forceinline__ bool dig(const uint8_t* t, int n) {
  for (int i = 0; i < n; ++i)
    if (static_cast<uint32_t>(t[i] - '0') > 9u) return false;
  return true;
}
__device__ __forceinline__ int num2(const uint8_t* t) { return (t[0] - '0') * 10 + (t[1] - '0'); }
__device__ __forceinline__ int num4(const uint8_t* t) { return num2(t) * 100 + num2(t + 2); }

__device__ __forceinline__ int conv_integer(const uint8_t* t, int n, bool is32, uint64_t* out) {
  int i = 0;
  const bool neg = t[0] == '-';
  if (neg) i = 1;
  if (i >= n) return kConvFail;
  // leading zeros add nothing; up to 19 significant digits accumulate in 64
  // bits without overflow (10^19 < 2^64), and more exceed every limit
  while (i + 1 < n && t[i] == '0') ++i;
  if (n - i > 19) return kConvFail;
  uint64_t m = 0;
  for (; i < n; ++i) {
    const uint32_t d = static_cast<uint32_t>(t[i]) - '0';
    if (d > 9u) return kConvFail;
    m = m * 10 + d;
  }
  const uint64_t lim = is32 ? (neg ? 2147483648ull : 2147483647ull)
                            : (neg ? 9223372036854775808ull : 9223372036854775807ull);
  if (m > lim) return kConvFail;
  const uint64_t v = neg ? (0ull - m) : m;
  *out = is32 ? static_cast<uint64_t>(static_cast<uint32_t>(v)) : v;
  return kConvOk;
}

// -?d+(.d+)? with a decimal significand below 2^53 and at most 22 fraction
// digits: the significand and 10^k are exact doubles, so one IEEE division
// gives the correctly rounded value (Clinger's fast path).
__device__ __forceinline__ int conv_float64(const uint8_t* t, int n, uint64_t* out) {
  int i = 0;
  const bool neg = t[0] == '-';
  if (neg) i = 1;
  int intd = 0, frac = 0;
  bool dot = false;
  uint64_t m = 0;
  for (; i < n; ++i) {
    const uint8_t ch = t[i];
    if (ch == '.') {
      if (dot || intd == 0) return kConvFail;
      dot = true;
      continue;
    }
    const uint32_t d = static_cast<uint32_t>(ch) - '0';
    if (d > 9u) return kConvFail;
    m = m * 10 + d;
    if (m >= (1ull << 53)) return kConvFail;
    if (dot) ++frac; else ++intd;
  }
  if (intd == 0 || (dot && frac == 0) || frac > 22) return kConvFail;
  double v = static_cast<double>(m) / kPow10[frac];
  if (neg) v = -v;
  *out = static_cast<uint64_t>(__double_as_longlong(v));
  return kConvOk;
}

__device__ __forceinline__ int conv_date(const uint8_t* t, int n, uint64_t* out) {
  if (n != 10 || t[4] != '-' || t[7] != '-' || !dig(t, 4) || !dig(t + 5, 2) || !dig(t + 8, 2))
    return kConvFail;
  const int y = num4(t), m = num2(t + 5), d = num2(t + 8);
  if (!valid_date(y, m, d)) return kConvFail;
  *out = static_cast<uint64_t>(static_cast<uint32_t>(static_cast<int32_t>(days_since_epoch(y, m, d))));
  return kConvOk;
}

__device__ __forceinline__ int conv_timestamp(const uint8_t* t, int n, uint64_t* out) {
  if (n != 19 || t[4] != '-' || t[7] != '-' || (t[10] != ' ' && t[10] != 'T') || t[13] != ':' ||
      t[16] != ':')
    return kConvFail;
  if (!dig(t, 4) || !dig(t + 5, 2) || !dig(t + 8, 2) || !dig(t + 11, 2) || !dig(t + 14, 2) ||
      !dig(t + 17, 2))
    return kConvFail;
  const int y = num4(t), mo = num2(t + 5), d = num2(t + 8);
  const int hh = num2(t + 11), mi = num2(t + 14), ss = num2(t + 17);
  if (!valid_date(y, mo, d) || hh > 23 || mi > 59 || ss > 59) return kConvFail;
  *out = static_cast<uint64_t>(days_since_epoch(y, mo, d) * 86400 + hh * 3600 + mi * 60 + ss);
  return kConvOk;
}

// dd/Mon/yyyy:hh:mm:ss +hhmm
__device__ __forceinline__ int conv_clf(const uint8_t* t, int n, uint64_t* out) {
  if (n != 26 || t[2] != '/' || t[6] != '/' || t[11] != ':' || t[14] != ':' || t[17] != ':' ||
      t[20] != ' ' || (t[21] != '+' && t[21] != '-'))
    return kConvFail;
  if (!dig(t, 2) || !dig(t + 7, 4) || !dig(t + 12, 2) || !dig(t + 15, 2) || !dig(t + 18, 2) ||
      !dig(t + 22, 4))
    return kConvFail;
  const uint32_t name = t[3] | (t[4] << 8) | (t[5] << 16);
  int mo = 0;
  for (int k = 0; k < 12; ++k)
    if (kMonthNames[k] == name) mo = k + 1;
  const int d = num2(t), y = num4(t + 7), hh = num2(t + 12), mi = num2(t + 15), ss = num2(t + 18);
  const int oh = num2(t + 22), om = num2(t + 24);
  if (mo == 0 || !valid_date(y, mo, d) || hh > 23 || mi > 59 || ss > 59 || oh > 23 || om > 59)
    return kConvFail;
  const int64_t local = days_since_epoch(y, mo, d) * 86400 + hh * 3600 + mi * 60 + ss;
  const int64_t off = static_cast<int64_t>(oh) * 3600 + om * 60;
  *out = static_cast<uint64_t>(t[21] == '+' ? local - off : local + off);
  return kConvOk;
}

__device__ __forceinline__ int convert_value(uint32_t type, const uint8_t* t, int n, uint64_t* out) {
  *out = 0;
  if (n == 0) return kConvEmpty;
  if (n > kNumericMaxLen) return kConvFail;
  int st = kConvFail;
  switch (type) {
    case PP_INT32: st = conv_integer(t, n, true, out); break;
    case PP_INT64: st = conv_integer(t, n, false, out); break;
    case PP_FLOAT64: st = conv_float64(t, n, out); break;
    case PP_DATE_D: st = conv_date(t, n, out); break;
    case PP_TIMESTAMP_S: st = conv_timestamp(t, n, out); break;
    case PP_TIMESTAMP_CLF: st = conv_clf(t, n, out); break;
    default: break;
  }
  if (st != kConvOk) *out = 0;
  return st;
}

}  // namespace pp
