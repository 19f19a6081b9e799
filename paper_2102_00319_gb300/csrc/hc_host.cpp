// Host-side arithmetic of libhecnn: prime chain, Shoup constants, the
// discrete-Gaussian table, FP64 canonical-embedding FFTs and the centred CRT
// lift.  Built with -ffp-contract=off so every double operation is the
// correctly rounded IEEE one on x86-64 and aarch64 alike.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "hc_internal.h"

typedef unsigned __int128 u128;

namespace hch {

u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 powmod(u64 a, u64 e, u64 q) {
  u64 r = 1 % q;
  a %= q;
  for (; e; e >>= 1) {
    if (e & 1) r = mulmod(r, a, q);
    a = mulmod(a, a, q);
  }
  return r;
}

u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// Miller-Rabin with the twelve smallest primes as witnesses: deterministic
// for all 64-bit inputs.
bool is_prime(u64 n) {
  const u64 witnesses[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : witnesses) {
    if (n == p) return true;
    if (n % p == 0) return false;
  }
  u64 d = n - 1;
  int s = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++s;
  }
  for (u64 a : witnesses) {
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int r = 1; r < s && witness; ++r) {
      x = mulmod(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

// For each size in order, the largest unused prime p < 2^bits, p = 1 mod 2N.
int gen_primes(int log_n, const int* bits, int n, u64* out) {
  const u64 step = (u64)2 << log_n;
  for (int i = 0; i < n; ++i) {
    const int b = bits[i];
    if (b < log_n + 2 || b > 61) return -1;
    const u64 hi = (u64)1 << b, lo = hi >> 1;
    bool found = false;
    for (u64 c = hi - step + 1; c > lo; c -= step) {
      bool taken = false;
      for (int k = 0; k < i; ++k) taken |= (out[k] == c);
      if (!taken && is_prime(c)) {
        out[i] = c;
        found = true;
        break;
      }
    }
    if (!found) return -1;
  }
  return 0;
}

u64 primitive_2n_root(int log_n, u64 q) {
  const u64 two_n = (u64)2 << log_n;
  for (u64 g = 2; g < q; ++g) {
    u64 r = powmod(g, (q - 1) / two_n, q);
    if (powmod(r, two_n >> 1, q) == q - 1) return r;
  }
  return 0;
}

int bit_reverse(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// ------------------------------------------------------------------------
// Double-double arithmetic (Dekker / Knuth error-free transforms; the
// product error term by a correctly rounded fma) for the Gaussian table.
// ------------------------------------------------------------------------
namespace {
struct DD {
  double hi, lo;
};
DD two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
DD quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
DD dd_add(DD a, DD b) {
  DD s = two_sum(a.hi, b.hi);
  DD t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
DD dd_mul(DD a, DD b) {
  double p = a.hi * b.hi;
  double e = std::fma(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p, e);
}
DD dd_div(DD a, DD b) {
  double q1 = a.hi / b.hi;
  DD r = dd_add(a, dd_mul(b, DD{-q1, 0.0}));
  double q2 = r.hi / b.hi;
  r = dd_add(r, dd_mul(b, DD{-q2, 0.0}));
  double q3 = r.hi / b.hi;
  DD q = quick_two_sum(q1, q2);
  return dd_add(q, DD{q3, 0.0});
}
// exp(-x), x >= 0: Taylor series of exp(-x / 2^12), then 12 squarings.
DD dd_exp_neg(DD x) {
  DD y = dd_mul(x, DD{-1.0 / 4096.0, 0.0});
  DD term{1.0, 0.0}, sum{1.0, 0.0};
  for (int k = 1; k < 30; ++k) {
    term = dd_div(dd_mul(term, y), DD{(double)k, 0.0});
    sum = dd_add(sum, term);
  }
  for (int i = 0; i < 12; ++i) sum = dd_mul(sum, sum);
  return sum;
}
}  // namespace

// cdt[k] = floor(2^63 Pr[|X| <= k]) for the discrete Gaussian with
// parameter sigma (the exact double), tail cut floor(6 sigma).
std::vector<u64> gaussian_cdt(double sigma) {
  const int tail = (int)std::floor(6.0 * sigma);
  DD s2 = dd_mul(DD{sigma, 0.0}, DD{sigma, 0.0});
  DD two_s2 = dd_mul(s2, DD{2.0, 0.0});
  std::vector<DD> rho(tail + 1);
  for (int k = 0; k <= tail; ++k) rho[k] = dd_exp_neg(dd_div(DD{(double)k * k, 0.0}, two_s2));
  DD z = rho[0];
  for (int k = 1; k <= tail; ++k) z = dd_add(z, dd_mul(rho[k], DD{2.0, 0.0}));
  std::vector<u64> out;
  DD cum{0.0, 0.0};
  for (int k = 0; k < tail; ++k) {
    DD p = k == 0 ? rho[0] : dd_mul(rho[k], DD{2.0, 0.0});
    cum = dd_add(cum, dd_div(p, z));
    DD v = dd_mul(cum, DD{9223372036854775808.0, 0.0});  // 2^63
    double fh = std::floor(v.hi);
    double r = (v.hi - fh) + v.lo;  // v.hi - fh is exact
    u64 t = (u64)fh;
    double fr = std::floor(r);
    if (fr < 0) t -= (u64)(-fr);
    else t += (u64)fr;
    out.push_back(t);
  }
  return out;
}

int64_t round_half_away(double x, bool* ok) {
  *ok = std::fabs(x) < 4611686018427387904.0;  // 2^62
  if (!*ok) return 0;
  return (int64_t)std::llround(x);
}

// ------------------------------------------------------------------------
// Canonical embedding by FFT.  Slot j sits at the odd exponent
// k_j = 5^j mod 2N (conjugate at -k_j).  With k = 2t + 1:
//   encode: m_i = Re( (scale/N) zeta^{-i} sum_t v_t omega^{-t i} ),
//   decode: m(zeta^{2t+1}) = sum_i (m_i zeta^i) omega^{t i},
// omega = zeta^2 = exp(2 pi i / N).
// ------------------------------------------------------------------------
namespace {
typedef std::complex<double> cd;

void fft(std::vector<cd>& a, bool inverse) {
  const size_t n = a.size();
  int bits = 0;
  while (((size_t)1 << bits) < n) ++bits;
  for (size_t i = 0; i < n; ++i) {
    size_t j = (size_t)bit_reverse((int)i, bits);
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t half = len >> 1, step = n / len;
    for (size_t i = 0; i < n; i += len)
      for (size_t k = 0; k < half; ++k) {
        const double ang = 2.0 * M_PI * (double)(k * step) / (double)n;
        cd w(std::cos(ang), inverse ? -std::sin(ang) : std::sin(ang));
        cd u = a[i + k], v = a[i + k + half] * w;
        a[i + k] = u + v;
        a[i + k + half] = u - v;
      }
  }
}

cd zeta_pow(long long e, int log_n) {
  const long long two_n = 2LL << log_n;
  e %= two_n;
  if (e < 0) e += two_n;
  const double ang = M_PI * (double)e / (double)(1LL << log_n);
  return cd(std::cos(ang), std::sin(ang));
}
}  // namespace

void encode_coeffs(const double* re, const double* im, size_t n_slots, int log_n, double scale,
                   std::vector<double>& coeffs) {
  const size_t n = (size_t)1 << log_n, K = n / 2, two_n = 2 * n;
  std::vector<cd> v(n, cd(0, 0));
  u64 g = 1;
  for (size_t j = 0; j < K; ++j) {
    cd z = j < n_slots ? cd(re[j], im ? im[j] : 0.0) : cd(0, 0);
    v[(g - 1) / 2] = z;
    v[(two_n - g - 1) / 2] = std::conj(z);
    g = (g * 5) % two_n;
  }
  fft(v, true);
  coeffs.assign(n, 0.0);
  for (size_t i = 0; i < n; ++i) {
    cd t = v[i] * zeta_pow(-(long long)i, log_n);
    coeffs[i] = t.real() * (scale / (double)n);
  }
}

void decode_slots(const std::vector<double>& coeffs, int log_n, double scale, double* re,
                  double* im, size_t n_out) {
  const size_t n = (size_t)1 << log_n, K = n / 2, two_n = 2 * n;
  std::vector<cd> v(n);
  for (size_t i = 0; i < n; ++i) v[i] = coeffs[i] * zeta_pow((long long)i, log_n);
  fft(v, false);
  u64 g = 1;
  for (size_t j = 0; j < K && j < n_out; ++j) {
    cd z = v[(g - 1) / 2] / scale;
    re[j] = z.real();
    if (im) im[j] = z.imag();
    g = (g * 5) % two_n;
  }
}

// ------------------------------------------------------------------------
// Centred CRT lift to double with multiword integers (little-endian words).
// ------------------------------------------------------------------------
namespace {
typedef std::vector<u64> Big;

Big big_mul_small(const Big& a, u64 m) {
  Big r(a.size() + 1, 0);
  u64 carry = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    u128 p = (u128)a[i] * m + carry;
    r[i] = (u64)p;
    carry = (u64)(p >> 64);
  }
  r[a.size()] = carry;
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  return r;
}
// a += b * m (a sized to hold the result)
void big_addmul(Big& a, const Big& b, u64 m) {
  u64 carry = 0;
  size_t i = 0;
  for (; i < b.size(); ++i) {
    u128 p = (u128)b[i] * m + a[i] + carry;
    a[i] = (u64)p;
    carry = (u64)(p >> 64);
  }
  for (; carry && i < a.size(); ++i) {
    u128 p = (u128)a[i] + carry;
    a[i] = (u64)p;
    carry = (u64)(p >> 64);
  }
}
int big_cmp(const Big& a, const Big& b) {  // same length
  for (size_t i = a.size(); i-- > 0;) {
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  }
  return 0;
}
void big_sub(Big& a, const Big& b) {  // a -= b, a >= b, same length
  u64 borrow = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    u128 s = (u128)a[i] - b[i] - borrow;
    a[i] = (u64)s;
    borrow = (u64)(s >> 64) ? 1 : 0;
  }
}
double big_to_double(const Big& a) {
  double r = 0.0;
  for (size_t i = a.size(); i-- > 0;) r = r * 18446744073709551616.0 + (double)a[i];
  return r;
}
}  // namespace

void crt_centred_to_double(const u64* res, const u64* primes, int nl, int n,
                           std::vector<double>& out) {
  out.assign((size_t)n, 0.0);
  Big Q{1};
  for (int l = 0; l < nl; ++l) Q = big_mul_small(Q, primes[l]);
  const size_t W = Q.size() + 2;
  Q.resize(W, 0);
  std::vector<Big> hat(nl);
  std::vector<u64> hat_inv(nl);
  for (int l = 0; l < nl; ++l) {
    Big h{1};
    u64 hm = 1;
    for (int k = 0; k < nl; ++k)
      if (k != l) {
        h = big_mul_small(h, primes[k]);
        hm = mulmod(hm, primes[k] % primes[l], primes[l]);
      }
    h.resize(W, 0);
    hat[l] = h;
    hat_inv[l] = invmod(hm, primes[l]);
  }
  Big half(W, 0);  // floor(Q / 2)
  for (size_t i = 0; i < W; ++i) half[i] = (Q[i] >> 1) | (i + 1 < W ? (Q[i + 1] << 63) : 0);
  Big x(W);
  for (int c = 0; c < n; ++c) {
    std::fill(x.begin(), x.end(), 0);
    for (int l = 0; l < nl; ++l) big_addmul(x, hat[l], mulmod(res[(size_t)l * n + c], hat_inv[l], primes[l]));
    while (big_cmp(x, Q) >= 0) big_sub(x, Q);
    if (big_cmp(x, half) > 0) {
      Big y = Q;
      big_sub(y, x);
      out[c] = -big_to_double(y);
    } else {
      out[c] = big_to_double(x);
    }
  }
}

}  // namespace hch
