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

#include <cmath>
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

// local vertices of face f (the three vertices other than f, increasing)
constexpr int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
// face orientation codes: own face vertex x <-> neighbour face vertex kPerm[c][x]
constexpr int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Packed connectivity word per (element, face): (nb << 5) | (nface << 3) | perm,
// or -1 on a wall. Limits the mesh to 2^26 elements.
constexpr int64_t kMaxElements = int64_t(1) << 26;

// Packed stencil words. A one-degree reduction (E^n_{n-1})^T produces output
// beta (degree n-1) from inputs beta + e_m (degree n) at
//   base, base + 1, base + dk, base + dl,   base = idx3(n, j, k, l),
//   dk = n - l - k + 1,  dl = (n-l+1)(n-l+2)/2 - k,
// with weights (beta_0+1, j+1, k+1, l+1) / n where beta_0 + 1 = n + 3 - the
// other three. A one-degree elevation E^n_{n-1} produces output gamma (degree
// n) from gamma - e_m (degree n-1) at base, base - 1, base - dk, base - dl,
// base = idx3(n-1, j, k, l) (a virtual index when gamma_0 = 0, whose term has
// weight 0), the same dk, dl, and weights (gamma_0, j, k, l) / n.
// Word: base (9 bits) | dk (4) | dl (7) | w1 (4) | w2 (4) | w3 (4).
BBW_HD constexpr uint32_t pack_stencil3(int base, int dk, int dl, int w1, int w2, int w3) {
  return uint32_t(base) | (uint32_t(dk) << 9) | (uint32_t(dl) << 13) | (uint32_t(w1) << 20) |
         (uint32_t(w2) << 24) | (uint32_t(w3) << 28);
}
// 2D analogue on a face: inputs base, base + 1, base + db (reduction) or
// base, base - 1, base - db (elevation); db = n + 1 - b2 for a reduction from
// degree n, db = n - a2 + 1 for an elevation to degree n.
// Word: base (7 bits) | db (4) | w1 (4) | w2 (4).
BBW_HD constexpr uint32_t pack_stencil2(int base, int db, int w1, int w2) {
  return uint32_t(base) | (uint32_t(db) << 7) | (uint32_t(w1) << 11) | (uint32_t(w2) << 15);
}

// Offset of pyramid level i in the per-face lift buffer: level i holds the
// np2(N - i) coefficients of degree N - i, levels stacked from i = 0, so that
// the whole pyramid of one face fills np3(N) slots.
BBW_HD constexpr int lift_level_base(int N, int i) { return np3(N) - np3(N - i); }

// Operator tables for one (N, M, real). Plain data, built on the host by
// build_tables(), copied once to device memory and from there into each
// CTA's shared memory.
template <int N, int M, typename real>
struct Tables {
  static constexpr int Np = np3(N);
  static constexpr int Nfp = np2(N);
  static constexpr int Mp = np3(M);
  static constexpr int NMp = np3(N + M);

  real invfactN[Np + 1];  // 1 / alpha!        (degree N; pad entry 0)
  real factNM[NMp];       // gamma! / C(N+M,N)  (degree N+M)
  real invfactM[Mp];      // 1 / beta!          (degree M)
  real cj[N + 1];         // projection constants c_j of Theorem 5.3
  // lift: level i of a face pyramid is stored scaled by ell_i = (-1)^i C(N,i)/(i+1);
  // lscale[i] = ell_i / (ell_{i-1} (N - i + 1)) turns a 2D reduction of the
  // stored level i - 1 (integer weights) into the stored level i (i >= 1)
  real lscale[N + 1];
  uint32_t red3[off3(N + M)];   // reduction words, outputs of degree d = 0..N+M-1
  uint32_t elev3[off3(N + 1)];  // elevation words, outputs of degree n = 0..N
  uint32_t red2[off2(N)];       // 2D reduction words, outputs of degree 0..N-1
  uint32_t elev2[np2(N)];       // 2D elevation words, outputs of degree N
  static constexpr int MP2 = (Mp + 1) / 2;
  // product gather: word [p][gamma] holds the degree-N indices of gamma-beta
  // for beta = 2p (low 16 bits) and 2p+1 (high), Np where gamma !>= beta
  uint32_t prod2[MP2 * NMp];
  uint16_t fidx[4 * Nfp];       // own volume index of face node a of face f
  uint16_t nidx[24 * Nfp];      // neighbour volume index for (nface, perm, a)
  // lift gather: for node i, byte f is the slot of its coefficient in the
  // pyramid of face f, lift_level_base(N, alpha_f) + idx2(N - alpha_f, .)
  uint32_t lgat[Np];
  static_assert(Np <= 256, "8-bit lift gather slots");
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
  // reductions into degree d from d + 1
  for (int d = 0; d < N + M; ++d) {
    const int n = d + 1;
    int c = 0;
    for (int l = 0; l <= d; ++l)
      for (int k = 0; k <= d - l; ++k)
        for (int j = 0; j <= d - l - k; ++j)
          t.red3[off3(d) + c++] = pack_stencil3(idx3(n, j, k, l), n - l - k + 1,
                                                (n - l + 1) * (n - l + 2) / 2 - k, j + 1, k + 1, l + 1);
  }
  // elevations into degree n from n - 1
  for (int n = 1; n <= N; ++n) {
    int c = 0;
    for (int l = 0; l <= n; ++l)
      for (int k = 0; k <= n - l; ++k)
        for (int j = 0; j <= n - l - k; ++j)
          t.elev3[off3(n) + c++] = pack_stencil3(idx3(n - 1, j, k, l), n - l - k + 1,
                                                 (n - l + 1) * (n - l + 2) / 2 - k, j, k, l);
  }
  t.elev3[0] = 0;
  for (int d = 0; d < N; ++d) {
    const int n = d + 1;
    int c = 0;
    for (int b2 = 0; b2 <= d; ++b2)
      for (int b1 = 0; b1 <= d - b2; ++b1)
        t.red2[off2(d) + c++] = pack_stencil2(idx2(n, b1, b2), n + 1 - b2, b1 + 1, b2 + 1);
  }
  {
    int c = 0;
    for (int a2 = 0; a2 <= N; ++a2)
      for (int a1 = 0; a1 <= N - a2; ++a1) t.elev2[c++] = pack_stencil2(idx2(N - 1, a1, a2), N - a2 + 1, a1, a2);
  }
  // multi-indices in the library order
  auto mi = [](int n, int i, int a[4]) {
    int c = 0;
    for (int l = 0; l <= n; ++l)
      for (int k = 0; k <= n - l; ++k)
        for (int j = 0; j <= n - l - k; ++j, ++c)
          if (c == i) {
            a[0] = n - j - k - l;
            a[1] = j;
            a[2] = k;
            a[3] = l;
            return;
          }
  };
  auto mi2 = [](int n, int i, int b[3]) {
    int c = 0;
    for (int b2 = 0; b2 <= n; ++b2)
      for (int b1 = 0; b1 <= n - b2; ++b1, ++c)
        if (c == i) {
          b[0] = n - b1 - b2;
          b[1] = b1;
          b[2] = b2;
          return;
        }
  };
  for (int i = 0; i < Tb::Np; ++i) {
    int a[4];
    mi(N, i, a);
    t.invfactN[i] = real(1.0 / (fact(a[0]) * fact(a[1]) * fact(a[2]) * fact(a[3])));
  }
  t.invfactN[Tb::Np] = real(0);
  const double cnm = binom(N + M, N);
  for (int i = 0; i < Tb::NMp; ++i) {
    int g[4];
    mi(N + M, i, g);
    t.factNM[i] = real(fact(g[0]) * fact(g[1]) * fact(g[2]) * fact(g[3]) / cnm);
    for (int b = 0; b < Tb::Mp; ++b) {
      int be[4];
      mi(M, b, be);
      bool ok = true;
      for (int x = 0; x < 4; ++x) ok = ok && g[x] >= be[x];
      const uint32_t src = uint32_t(ok ? idx3(N, g[1] - be[1], g[2] - be[2], g[3] - be[3]) : Tb::Np);
      uint32_t& w = t.prod2[(b / 2) * Tb::NMp + i];
      w = (b & 1) ? (w & 0xffffu) | (src << 16) : src;
    }
    if (Tb::Mp & 1) t.prod2[(Tb::Mp / 2) * Tb::NMp + i] |= uint32_t(Tb::Np) << 16;
  }
  for (int b = 0; b < Tb::Mp; ++b) {
    int be[4];
    mi(M, b, be);
    t.invfactM[b] = real(1.0 / (fact(be[0]) * fact(be[1]) * fact(be[2]) * fact(be[3])));
  }
  auto ell = [&](int i) { return ((i & 1) ? -1.0 : 1.0) * binom(N, i) / (i + 1); };
  for (int j = 0; j <= N; ++j) {
    t.cj[j] = real(cj[j]);
    t.lscale[j] = j == 0 ? real(1) : real(ell(j) / (ell(j - 1) * (N - j + 1)));
  }
  for (int f = 0; f < 4; ++f) {
    for (int a = 0; a < Tb::Nfp; ++a) {
      int b[3];
      mi2(N, a, b);
      int al[4] = {0, 0, 0, 0};
      for (int x = 0; x < 3; ++x) al[kFaceVerts[f][x]] = b[x];
      t.fidx[f * Tb::Nfp + a] = uint16_t(idx3(N, al[1], al[2], al[3]));
      for (int p = 0; p < 6; ++p) {
        int an[4] = {0, 0, 0, 0};
        for (int x = 0; x < 3; ++x) an[kFaceVerts[f][kPerm[p][x]]] = b[x];
        t.nidx[(f * 6 + p) * Tb::Nfp + a] = uint16_t(idx3(N, an[1], an[2], an[3]));
      }
    }
  }
  // lift gather slots
  for (int i = 0; i < Tb::Np; ++i) {
    int a[4];
    mi(N, i, a);
    uint32_t w = 0;
    for (int f = 0; f < 4; ++f) {
      int b[3];
      for (int x = 0; x < 3; ++x) b[x] = a[kFaceVerts[f][x]];
      w |= uint32_t(lift_level_base(N, a[f]) + idx2(N - a[f], b[1], b[2])) << (8 * f);
    }
    t.lgat[i] = w;
  }
}

// Host-side check of a built table set against brute force: every stencil
// word, product index, face map and lift slot is recomputed from the lattice
// enumeration (not from idx3 / idx2) and range-checked. Returns nullptr if
// all entries agree, else a description of the first mismatch.
template <int N, int M, typename real>
const char* validate_tables(const Tables<N, M, real>& t) {
  using Tb = Tables<N, M, real>;
  // position of multi-index (j, k, l) of degree n, by enumeration
  auto pos3 = [](int n, int j, int k, int l) {
    if (j < 0 || k < 0 || l < 0 || j + k + l > n) return -1;
    int c = 0;
    for (int ll = 0; ll <= n; ++ll)
      for (int kk = 0; kk <= n - ll; ++kk)
        for (int jj = 0; jj <= n - ll - kk; ++jj, ++c)
          if (jj == j && kk == k && ll == l) return c;
    return -1;
  };
  auto pos2 = [](int n, int b1, int b2) {
    if (b1 < 0 || b2 < 0 || b1 + b2 > n) return -1;
    int c = 0;
    for (int bb2 = 0; bb2 <= n; ++bb2)
      for (int bb1 = 0; bb1 <= n - bb2; ++bb1, ++c)
        if (bb1 == b1 && bb2 == b2) return c;
    return -1;
  };
  auto s3 = [](uint32_t w, int f) {
    const int v[6] = {int(w & 511u), int((w >> 9) & 15u), int((w >> 13) & 127u), int((w >> 20) & 15u),
                      int((w >> 24) & 15u), int(w >> 28)};
    return v[f];
  };
  auto s2 = [](uint32_t w, int f) {
    const int v[4] = {int(w & 127u), int((w >> 7) & 15u), int((w >> 11) & 15u), int((w >> 15) & 15u)};
    return v[f];
  };
  // one-degree reductions into degree d: inputs beta + e_m of degree d + 1
  for (int d = 0; d < N + M; ++d) {
    const int n = d + 1;
    int c = 0;
    for (int l = 0; l <= d; ++l)
      for (int k = 0; k <= d - l; ++k)
        for (int j = 0; j <= d - l - k; ++j, ++c) {
          const uint32_t w = t.red3[off3(d) + c];
          const int b = s3(w, 0);
          if (b != pos3(n, j, k, l) || b + 1 != pos3(n, j + 1, k, l) || b + s3(w, 1) != pos3(n, j, k + 1, l) ||
              b + s3(w, 2) != pos3(n, j, k, l + 1))
            return "reduction stencil offsets";
          if (s3(w, 3) != j + 1 || s3(w, 4) != k + 1 || s3(w, 5) != l + 1) return "reduction stencil weights";
        }
  }
  // one-degree elevations into degree n: inputs gamma - e_m of degree n - 1
  for (int n = 1; n <= N; ++n) {
    int c = 0;
    for (int l = 0; l <= n; ++l)
      for (int k = 0; k <= n - l; ++k)
        for (int j = 0; j <= n - l - k; ++j, ++c) {
          const uint32_t w = t.elev3[off3(n) + c];
          const int b = s3(w, 0), g0 = n - j - k - l;
          if (s3(w, 3) != j || s3(w, 4) != k || s3(w, 5) != l) return "elevation stencil weights";
          if ((g0 > 0 && b != pos3(n - 1, j, k, l)) || (j > 0 && b - 1 != pos3(n - 1, j - 1, k, l)) ||
              (k > 0 && b - s3(w, 1) != pos3(n - 1, j, k - 1, l)) ||
              (l > 0 && b - s3(w, 2) != pos3(n - 1, j, k, l - 1)))
            return "elevation stencil offsets";
        }
  }
  for (int d = 0; d < N; ++d) {
    const int n = d + 1;
    int c = 0;
    for (int b2 = 0; b2 <= d; ++b2)
      for (int b1 = 0; b1 <= d - b2; ++b1, ++c) {
        const uint32_t w = t.red2[off2(d) + c];
        const int b = s2(w, 0);
        if (b != pos2(n, b1, b2) || b + 1 != pos2(n, b1 + 1, b2) || b + s2(w, 1) != pos2(n, b1, b2 + 1))
          return "2D reduction stencil offsets";
        if (s2(w, 2) != b1 + 1 || s2(w, 3) != b2 + 1) return "2D reduction stencil weights";
      }
  }
  {
    int c = 0;
    for (int a2 = 0; a2 <= N; ++a2)
      for (int a1 = 0; a1 <= N - a2; ++a1, ++c) {
        const uint32_t w = t.elev2[c];
        const int b = s2(w, 0), a0 = N - a1 - a2;
        if (s2(w, 2) != a1 || s2(w, 3) != a2) return "2D elevation stencil weights";
        if ((a0 > 0 && b != pos2(N - 1, a1, a2)) || (a1 > 0 && b - 1 != pos2(N - 1, a1 - 1, a2)) ||
            (a2 > 0 && b - s2(w, 1) != pos2(N - 1, a1, a2 - 1)))
          return "2D elevation stencil offsets";
      }
  }
  // product gather: gamma - beta in the degree-N lattice, Np where gamma !>= beta
  {
    int c = 0;
    for (int l = 0; l <= N + M; ++l)
      for (int k = 0; k <= N + M - l; ++k)
        for (int j = 0; j <= N + M - l - k; ++j, ++c) {
          int b = 0;
          for (int bl = 0; bl <= M; ++bl)
            for (int bk = 0; bk <= M - bl; ++bk)
              for (int bj = 0; bj <= M - bl - bk; ++bj, ++b) {
                const int g0 = N + M - j - k - l, b0 = M - bj - bk - bl;
                int want = g0 >= b0 ? pos3(N, j - bj, k - bk, l - bl) : -1;
                if (want < 0) want = Tb::Np;
                const uint32_t w = t.prod2[(b / 2) * Tb::NMp + c];
                const int got = int((b & 1) ? (w >> 16) : (w & 0xffffu));
                if (got != want) return "product gather index";
              }
        }
  }
  // face maps and lift gather slots
  for (int i = 0; i < 4 * Tb::Nfp; ++i)
    if (t.fidx[i] >= Tb::Np) return "own face index out of range";
  for (int i = 0; i < 24 * Tb::Nfp; ++i)
    if (t.nidx[i] >= Tb::Np) return "neighbour face index out of range";
  {
    int c = 0;
    for (int l = 0; l <= N; ++l)
      for (int k = 0; k <= N - l; ++k)
        for (int j = 0; j <= N - l - k; ++j, ++c) {
          const int a[4] = {N - j - k - l, j, k, l};
          for (int f = 0; f < 4; ++f) {
            const int slot = int((t.lgat[c] >> (8 * f)) & 255u);
            if (slot < lift_level_base(N, a[f]) || slot >= lift_level_base(N, a[f] + 1))
              return "lift gather slot outside its level";
          }
        }
  }
  for (int i = 0; i <= N; ++i)
    if (!(t.cj[i] == t.cj[i]) || !(t.lscale[i] != real(0))) return "projection or lift constants";
  return nullptr;
}

}  // namespace bbw
