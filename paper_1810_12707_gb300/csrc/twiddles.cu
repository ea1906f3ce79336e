// twiddles.cu -- host construction of the twiddle tables the transforms read.
#include <math.h>
#include <string.h>

#include <vector>

#include "mhd_internal.h"

namespace mhd {

namespace {
const long double kTwoPi = 6.283185307179586476925286766559005768L;
}

// W_N^m = exp(-2 pi i m / N) for m < N, from first-octant values and exact quarter-turn
// symmetries, so that W^{N/4} = -i, W^{N/2} = -1 and W^{3N/4} = i hold exactly.
std::vector<cplx64> twiddle_table(int n) {
  const int q4 = n / 4, q8 = n / 8;
  std::vector<long double> C(q8 + 1), Sn(q8 + 1);
  for (int r = 0; r <= q8; ++r) {
    C[r] = cosl(kTwoPi * r / n);
    Sn[r] = sinl(kTwoPi * r / n);
  }
  C[0] = 1.0L;
  Sn[0] = 0.0L;
  std::vector<cplx64> w(n);
  for (int m = 0; m < n; ++m) {
    const int quad = m / q4, r = m % q4;
    double cs, sn;
    if (r <= q8) {
      cs = (double)C[r];
      sn = (double)Sn[r];
    } else {
      cs = (double)Sn[q4 - r];
      sn = (double)C[q4 - r];
    }
    double c2 = cs, s2 = sn;  // rotate by quad quarter turns: angle + quad * pi/2
    if (quad == 1) { c2 = -sn; s2 = cs; }
    if (quad == 2) { c2 = -cs; s2 = -sn; }
    if (quad == 3) { c2 = sn; s2 = -cs; }
    w[m] = cplx64{c2, -s2};
  }
  return w;
}

// The FP64 table: the classic table above, then for every m the pair (c, t) and the byte q with
// W_N^m = i^q c (1 + i t), |t| <= 1.  With q' = the nearest integer to 4m/N, W_N^m =
// i^(-q') exp(2 pi i d / N), d = q' N/4 - m in [-N/8, N/8]: c = cos(2 pi d/N), t = tan(2 pi d/N).
std::vector<unsigned char> fp64_twiddle_bytes(int n) {
  const std::vector<cplx64> w = twiddle_table(n);
  std::vector<unsigned char> out(fp64_twiddle_size(n));
  memcpy(out.data(), w.data(), (size_t)n * sizeof(cplx64));
  double *ct = reinterpret_cast<double *>(out.data() + (size_t)n * sizeof(cplx64));
  unsigned char *q = out.data() + (size_t)n * 2 * sizeof(cplx64);
  for (int m = 0; m < n; ++m) {
    const int qr = (4 * m + n / 2) / n;  // nearest integer to 4m/N, 0..4
    const int d = qr * (n / 4) - m;      // -N/8 .. N/8
    const int ad = d < 0 ? -d : d;
    double c, t;
    if (d == 0) {
      c = 1.0;
      t = 0.0;
    } else if (8 * ad == n) {
      c = (double)cosl(kTwoPi / 8);
      t = d > 0 ? 1.0 : -1.0;
    } else {
      c = (double)cosl(kTwoPi * ad / n);
      t = (double)(tanl(kTwoPi * ad / n) * (d > 0 ? 1 : -1));
    }
    ct[2 * m] = c;
    ct[2 * m + 1] = t;
    q[m] = (unsigned char)((4 - qr) & 3);
  }
  return out;
}

}  // namespace mhd
