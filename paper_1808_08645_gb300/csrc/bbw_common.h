// bbw_common.h -- index arithmetic and per-(N, M) operator tables shared by the
// host setup code and the device kernels of libbbwadg.
//
// Multi-index order (the paper leaves it open, Sec. 2): for degree n,
//   for l in 0..n, for k in 0..n-l, for j in 0..n-l-k: alpha = (n-j-k-l, j, k, l)
// so that idx3(n, j, k, l) = P3(n) - P3(n-l) + k (n-l+1) - k (k-1) / 2 + j,
// with P3(m) = (m+1)(m+2)(m+3)/6 the dimension of P^m (the layers l' >= l form
// a degree n-l lattice). Triangle faces use (b0, b1, b2), b2 outer, b1 inner:
// idx2(n, b1, b2) = b2 (n+1) - b2 (b2-1) / 2 + b1.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define BBW_HD __host__ __device__ __forceinline__
#else
#define BBW_HD inline
#endif

namespace bbw {

constexpr int kMaxN = 9;
constexpr int kMaxM = 3;

BBW_HD constexpr int np3(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) * (n + 3) / 6; }
BBW_HD constexpr int np2(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) / 2; }
// sum_{m<n} np3(m) and sum_{m<n} np2(m): offsets of degree n in the
// concatenated decode tables.
BBW_HD constexpr int off3(int n) { return n * (n + 1) * (n + 2) * (n + 3) / 24; }
BBW_HD constexpr int off2(int n) { return n * (n + 1) * (n + 2) / 6; }

BBW_HD constexpr int idx3(int n, int j, int k, int l) {
  return np3(n) - np3(n - l) + k * (n - l + 1) - k * (k - 1) / 2 + j;
}
BBW_HD constexpr int idx2(int n, int b1, int b2) { return b2 * (n + 1) - b2 * (b2 - 1) / 2 + b1; }

BBW_HD constexpr uint32_t pack4(int a0, int a1, int a2, int a3) {
  return uint32_t(a0) | (uint32_t(a1) << 8) | (uint32_t(a2) << 16) | (uint32_t(a3) << 24);
}

// local vertices of face f (the three vertices other than f, increasing)
constexpr int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
// face orientation codes: own face vertex x <-> neighbour face vertex kPerm[c][x]
constexpr int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Packed connectivity word per (element, face): (nb << 5) | (nface << 3) | perm,
// or -1 on a wall. Limits the mesh to 2^26 elements.
constexpr int64_t kMaxElements = int64_t(1) << 26;

// Operator tables for one (N, M, real). Plain data, built on the host by
// build_tables(), copied once to device memory and from there into each
// CTA's shared memory.
template <int N, int M, typename real>
struct Tables {
  static constexpr int Np = np3(N);
  static constexpr int Nfp = np2(N);
  static constexpr int Mp = np3(M);
  static constexpr int NMp = np3(N + M);
  static constexpr int kDec3 = off3(N + M + 1);  // decode of degrees 0..N+M
  static constexpr int kDec2 = off2(N + 1);      // 2D decode of degrees 0..N

  real invfactN[Np + 1];  // 1 / alpha!        (degree N; pad entry unused)
  real factNM[NMp];       // gamma! / C(N+M,N)  (degree N+M)
  real invfactM[Mp];      // 1 / beta!          (degree M)
  real cj[N + 1];         // projection constants c_j of Theorem 5.3
  real ell[N + 1];        // lift layer factors (-1)^i C(N,i) / (i+1)
  uint32_t dec3[kDec3];   // packed alpha of each index, per degree
  uint32_t dec2[kDec2];   // packed (b0,b1,b2) of each 2D index, per degree
  uint16_t prod[NMp * Mp];  // index of gamma-beta in degree N, or Np if gamma !>= beta
  uint16_t fidx[4 * Nfp];   // own volume index of face node a of face f
  uint16_t nidx[24 * Nfp];  // neighbour volume index for (nface, perm, a)
  uint16_t lidx[4 * Np];    // volume index of (face f, layer i, face coords b)
};

template <int N, int M, typename real>
constexpr int table_bytes() {
  return int((sizeof(Tables<N, M, real>) + 15) / 16 * 16);
}

// Host-side construction of the tables. cj: the N+1 projection constants.
template <int N, int M, typename real>
void build_tables(Tables<N, M, real>& t, const double* cj) {
  using Tb = Tables<N, M, real>;
  auto fact = [](int n) {
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
  };
  auto binom = [&](int n, int k) { return fact(n) / (fact(k) * fact(n - k)); };
  for (int n = 0; n <= N + M; ++n) {
    int c = 0;
    for (int l = 0; l <= n; ++l)
      for (int k = 0; k <= n - l; ++k)
        for (int j = 0; j <= n - l - k; ++j) t.dec3[off3(n) + c++] = pack4(n - j - k - l, j, k, l);
  }
  for (int n = 0; n <= N; ++n) {
    int c = 0;
    for (int b2 = 0; b2 <= n; ++b2)
      for (int b1 = 0; b1 <= n - b2; ++b1) t.dec2[off2(n) + c++] = pack4(n - b1 - b2, b1, b2, 0);
  }
  auto unpack = [](uint32_t w, int a[4]) {
    for (int x = 0; x < 4; ++x) a[x] = int((w >> (8 * x)) & 255u);
  };
  for (int i = 0; i < Tb::Np; ++i) {
    int a[4];
    unpack(t.dec3[off3(N) + i], a);
    t.invfactN[i] = real(1.0 / (fact(a[0]) * fact(a[1]) * fact(a[2]) * fact(a[3])));
  }
  t.invfactN[Tb::Np] = real(0);
  const double cnm = binom(N + M, N);
  for (int i = 0; i < Tb::NMp; ++i) {
    int g[4];
    unpack(t.dec3[off3(N + M) + i], g);
    t.factNM[i] = real(fact(g[0]) * fact(g[1]) * fact(g[2]) * fact(g[3]) / cnm);
    for (int b = 0; b < Tb::Mp; ++b) {
      int be[4];
      unpack(t.dec3[off3(M) + b], be);
      bool ok = true;
      for (int x = 0; x < 4; ++x) ok = ok && g[x] >= be[x];
      t.prod[i * Tb::Mp + b] =
          uint16_t(ok ? idx3(N, g[1] - be[1], g[2] - be[2], g[3] - be[3]) : Tb::Np);
    }
  }
  for (int b = 0; b < Tb::Mp; ++b) {
    int be[4];
    unpack(t.dec3[off3(M) + b], be);
    t.invfactM[b] = real(1.0 / (fact(be[0]) * fact(be[1]) * fact(be[2]) * fact(be[3])));
  }
  for (int j = 0; j <= N; ++j) {
    t.cj[j] = real(cj[j]);
    t.ell[j] = real(((j & 1) ? -1.0 : 1.0) * binom(N, j) / (j + 1));
  }
  // face maps
  for (int f = 0; f < 4; ++f) {
    for (int a = 0; a < Tb::Nfp; ++a) {
      int b[4];
      unpack(t.dec2[off2(N) + a], b);
      int al[4] = {0, 0, 0, 0};
      for (int x = 0; x < 3; ++x) al[kFaceVerts[f][x]] = b[x];
      t.fidx[f * Tb::Nfp + a] = uint16_t(idx3(N, al[1], al[2], al[3]));
      for (int p = 0; p < 6; ++p) {
        int an[4] = {0, 0, 0, 0};
        for (int x = 0; x < 3; ++x) an[kFaceVerts[f][kPerm[p][x]]] = b[x];
        t.nidx[(f * 6 + p) * Tb::Nfp + a] = uint16_t(idx3(N, an[1], an[2], an[3]));
      }
    }
    int off = 0;
    for (int layer = 0; layer <= N; ++layer) {
      const int n2 = N - layer;
      for (int a = 0; a < np2(n2); ++a) {
        int b[4];
        unpack(t.dec2[off2(n2) + a], b);
        int al[4] = {0, 0, 0, 0};
        al[f] = layer;
        for (int x = 0; x < 3; ++x) al[kFaceVerts[f][x]] = b[x];
        t.lidx[f * Tb::Np + off + a] = uint16_t(idx3(N, al[1], al[2], al[3]));
      }
      off += np2(n2);
    }
  }
}

}  // namespace bbw
