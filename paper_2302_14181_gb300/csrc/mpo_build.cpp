// Host construction of the order-N time-evolution MPO W^(N)(tau)
// (arXiv:2302.14181, Secs. 2.5, 3-6; Algorithms 1-4; Eq. boundary).
//
// Levels of the N-th power of the Hamiltonian MPO are N-tuples over {1,2,3}
// (Sec. 2.5); here a level is packed two bits per copy (copy 0 in the lowest
// bits). An entry of the block matrix is a dense operator tensor stored as
// [v_left][d_out][d_in][v_right], v = chi^(number of 2s). The pipeline is
// H^N -> extension (Alg. 3, using H^(N+1)) -> fold (Alg. 1) -> exact
// compression (Alg. 2) -> approximate compression (Alg. 4), with the readings:
//   * Alg. 3 loops over the columns without a 1;
//   * "sort to the front" in Alg. 2 is a stable partition;
//   * Alg. 4 removes the levels that have a 3 and no 1, with factor
//     tau^n3 (N-n3)!/N!.
#include <algorithm>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "tevo_internal.h"

namespace tevo {

using cplx = std::complex<double>;

namespace {

struct Level {
  uint32_t code = 0;  // two bits per copy
  int n = 0;
  int at(int k) const { return int((code >> (2 * k)) & 3u); }
  void set(int k, int v) { code = (code & ~(3u << (2 * k))) | (uint32_t(v) << (2 * k)); }
  int count(int v) const {
    int c = 0;
    for (int k = 0; k < n; ++k) c += at(k) == v;
    return c;
  }
  bool operator<(const Level& o) const { return code < o.code; }
  bool operator==(const Level& o) const { return code == o.code && n == o.n; }
  bool operator!=(const Level& o) const { return !(*this == o); }
};

Level make_level(const std::vector<int>& v) {
  Level l;
  l.n = int(v.size());
  for (int k = 0; k < l.n; ++k) l.set(k, v[k]);
  return l;
}

std::vector<int> digits(const Level& l) {
  std::vector<int> v(l.n);
  for (int k = 0; k < l.n; ++k) v[k] = l.at(k);
  return v;
}

// tensor [vl][d][d][vr]
struct Op {
  int vl = 0, vr = 0, d = 0;
  std::vector<cplx> a;
  Op() = default;
  Op(int vl_, int d_, int vr_) : vl(vl_), vr(vr_), d(d_), a(size_t(vl_) * d_ * d_ * vr_) {}
  cplx& at(int i, int s, int t, int j) { return a[((size_t(i) * d + s) * d + t) * vr + j]; }
  cplx at(int i, int s, int t, int j) const { return a[((size_t(i) * d + s) * d + t) * vr + j]; }
  void axpy(cplx c, const Op& x) {
    for (size_t k = 0; k < a.size(); ++k) a[k] += c * x.a[k];
  }
};

struct Blocks {
  int chi, d;
  const double *A, *B, *C, *D;  // one site, interleaved complex
  cplx get(const double* p, size_t idx) const { return cplx(p[2 * idx], p[2 * idx + 1]); }
};

// single-copy transition block x -> y as [vl][d][d][vr]; returns false for zero
bool copy_op(const Blocks& b, int x, int y, Op& out) {
  const int d = b.d, chi = b.chi;
  if ((x == 1 && y == 1) || (x == 3 && y == 3)) {
    out = Op(1, d, 1);
    for (int s = 0; s < d; ++s) out.at(0, s, s, 0) = 1.0;
    return true;
  }
  if (x == 1 && y == 2) {  // C[k][s][t] -> [1][s][t][k]
    out = Op(1, d, chi);
    for (int k = 0; k < chi; ++k)
      for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t) out.at(0, s, t, k) = b.get(b.C, (size_t(k) * d + s) * d + t);
    return true;
  }
  if (x == 1 && y == 3) {
    out = Op(1, d, 1);
    for (int s = 0; s < d; ++s)
      for (int t = 0; t < d; ++t) out.at(0, s, t, 0) = b.get(b.D, size_t(s) * d + t);
    return true;
  }
  if (x == 2 && y == 2) {  // A[k][l][s][t] -> [k][s][t][l]
    out = Op(chi, d, chi);
    for (int k = 0; k < chi; ++k)
      for (int l = 0; l < chi; ++l)
        for (int s = 0; s < d; ++s)
          for (int t = 0; t < d; ++t)
            out.at(k, s, t, l) = b.get(b.A, ((size_t(k) * chi + l) * d + s) * d + t);
    return true;
  }
  if (x == 2 && y == 3) {  // B[k][s][t] -> [k][s][t][1]
    out = Op(chi, d, 1);
    for (int k = 0; k < chi; ++k)
      for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t) out.at(k, s, t, 0) = b.get(b.B, (size_t(k) * d + s) * d + t);
    return true;
  }
  return false;
}

// entry of the M-th power: operator product over copies (copy 0 leftmost),
// direct product on the virtual legs (copy 0 most significant)
bool power_op(const Blocks& b, const Level& a, const Level& c, Op& out) {
  const int d = b.d;
  Op P;
  for (int k = 0; k < a.n; ++k) {
    Op X;
    if (!copy_op(b, a.at(k), c.at(k), X)) return false;
    if (k == 0) {
      P = X;
      continue;
    }
    Op R(P.vl * X.vl, d, P.vr * X.vr);
    for (int i = 0; i < P.vl; ++i)
      for (int i2 = 0; i2 < X.vl; ++i2)
        for (int j = 0; j < P.vr; ++j)
          for (int j2 = 0; j2 < X.vr; ++j2)
            for (int s = 0; s < d; ++s)
              for (int u = 0; u < d; ++u) {
                cplx acc = 0;
                for (int t = 0; t < d; ++t) acc += P.at(i, s, t, j) * X.at(i2, t, u, j2);
                R.at(i * X.vl + i2, s, u, j * X.vr + j2) = acc;
              }
    P = std::move(R);
  }
  out = std::move(P);
  return true;
}

double factorial(int n) {
  double f = 1;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

struct BlockMatrix {
  int N, d, chi;
  std::vector<Level> alive;
  std::map<std::pair<uint32_t, uint32_t>, Op> ent;

  int vdim(const Level& l) const {
    int v = 1;
    for (int k = 0; k < l.count(2); ++k) v *= chi;
    return v;
  }
  bool has(const Level& a, const Level& b) const { return ent.count({a.code, b.code}) != 0; }
  Op& get(const Level& a, const Level& b) { return ent[{a.code, b.code}]; }
  void add(const Level& a, const Level& b, cplx c, const Op& x) {
    auto key = std::make_pair(a.code, b.code);
    auto it = ent.find(key);
    if (it == ent.end()) {
      Op z(x.vl, x.d, x.vr);
      z.axpy(c, x);
      ent.emplace(key, std::move(z));
    } else {
      it->second.axpy(c, x);
    }
  }
  void drop(const Level& c) {
    alive.erase(std::remove(alive.begin(), alive.end(), c), alive.end());
    for (auto it = ent.begin(); it != ent.end();) {
      if (it->first.first == c.code || it->first.second == c.code)
        it = ent.erase(it);
      else
        ++it;
    }
  }
  bool is_alive(const Level& c) const { return std::find(alive.begin(), alive.end(), c) != alive.end(); }
};

std::vector<Level> all_levels(int M) {
  std::vector<Level> out;
  int total = 1;
  for (int k = 0; k < M; ++k) total *= 3;
  for (int idx = 0; idx < total; ++idx) {
    std::vector<int> v(M);
    int r = idx;
    for (int k = M - 1; k >= 0; --k) {
      v[k] = 1 + r % 3;
      r /= 3;
    }
    out.push_back(make_level(v));
  }
  return out;
}

Level insert_at(const Level& a, int pos, int val) {
  std::vector<int> v = digits(a);
  v.insert(v.begin() + pos, val);
  return make_level(v);
}

Level stable_front(const Level& a, int val) {
  std::vector<int> v = digits(a), out;
  for (int x : v)
    if (x == val) out.push_back(x);
  for (int x : v)
    if (x != val) out.push_back(x);
  return make_level(out);
}

void build_site(const Blocks& blk, int N, cplx tau, int variant, std::vector<cplx>& W, int& w,
                std::vector<int>& offsets_out) {
  BlockMatrix O;
  O.N = N;
  O.d = blk.d;
  O.chi = blk.chi;
  O.alive = all_levels(N);
  for (const Level& a : O.alive)
    for (const Level& b : O.alive) {
      Op e;
      if (power_op(blk, a, b, e)) O.ent.emplace(std::make_pair(a.code, b.code), std::move(e));
    }
  const Level one = make_level(std::vector<int>(N, 1));

  // Algorithm 3: extension with the (N+1)-th power
  if (variant >= TEVO_MPO_EXTENDED) {
    std::vector<std::pair<std::pair<Level, Level>, Op>> upd;
    for (const Level& a : O.alive) {
      if (a.count(2) == 0 && a.count(3) > 0) continue;
      for (const Level& b : O.alive) {
        if (b.count(1) > 0) continue;
        Op acc;
        bool any = false;
        for (int c = 0; c <= N; ++c) {
          Level ae = insert_at(a, c, 1);
          for (int dp = 0; dp <= N; ++dp) {
            Level be = insert_at(b, dp, 3);
            Op e;
            if (!power_op(blk, ae, be, e)) continue;
            cplx coef = tau * factorial(N) / (factorial(N + 1) * ae.count(1) * be.count(3));
            if (!any) {
              acc = Op(e.vl, e.d, e.vr);
              any = true;
            }
            acc.axpy(coef, e);
          }
        }
        if (any) upd.push_back({{a, b}, std::move(acc)});
      }
    }
    for (auto& u : upd) O.add(u.first.first, u.first.second, 1.0, u.second);
  }

  // Algorithm 1: fold the pure {1,3} columns into (1,...,1)
  for (int a = 1; a <= N; ++a) {
    cplx coef = std::pow(tau, a) * factorial(N - a) / factorial(N);
    std::vector<int> base(N, 1);
    for (int k = 0; k < a; ++k) base[k] = 3;
    std::sort(base.begin(), base.end());
    do {
      Level b = make_level(base);
      for (const Level& r : O.alive)
        if (O.has(r, b)) {
          Op x = O.get(r, b);
          O.add(r, one, coef, x);
        }
      O.drop(b);
    } while (std::next_permutation(base.begin(), base.end()));
  }

  // Algorithm 2: exact compression
  if (variant >= TEVO_MPO_EXACT) {
    std::vector<Level> snapshot = O.alive;
    for (const Level& c : snapshot) {
      if (!O.is_alive(c)) continue;
      int n1 = c.count(1), n3 = c.count(3);
      Level sc = stable_front(c, 1), sr = stable_front(c, 3);
      if (n3 <= n1 && sc != c) {
        for (const Level& b : O.alive)
          if (O.has(c, b)) {
            Op x = O.get(c, b);
            O.add(sc, b, 1.0, x);
          }
        O.drop(c);
      } else if (n3 > n1 && sr != c) {
        for (const Level& r : O.alive)
          if (O.has(r, c)) {
            Op x = O.get(r, c);
            O.add(r, sr, 1.0, x);
          }
        O.drop(c);
      }
    }
  }

  // Algorithm 4: approximate compression
  if (variant >= TEVO_MPO_FULL) {
    std::vector<Level> snapshot = O.alive;
    for (const Level& a : snapshot) {
      if (a.count(1) > 0 || a.count(3) == 0) continue;
      int n3 = a.count(3);
      std::vector<int> v = digits(a);
      for (int& x : v)
        if (x == 3) x = 1;
      Level b = make_level(v);
      cplx coef = std::pow(tau, n3) * factorial(N - n3) / factorial(N);
      for (const Level& r : O.alive)
        if (O.has(r, a)) {
          Op x = O.get(r, a);
          O.add(r, b, coef, x);
        }
      O.drop(a);
    }
  }

  // dense W[w_l][s][s'][w_r], (1,...,1) first, then the others by code
  std::vector<Level> order;
  order.push_back(one);
  std::vector<Level> rest;
  for (const Level& l : O.alive)
    if (l != one) rest.push_back(l);
  std::sort(rest.begin(), rest.end());
  order.insert(order.end(), rest.begin(), rest.end());
  std::map<uint32_t, int> off;
  w = 0;
  offsets_out.clear();
  for (const Level& l : order) {
    off[l.code] = w;
    offsets_out.push_back(w);
    w += O.vdim(l);
  }
  const int d = blk.d;
  W.assign(size_t(w) * d * d * w, cplx(0));
  for (auto& kv : O.ent) {
    const Op& e = kv.second;
    int oa = off[kv.first.first], ob = off[kv.first.second];
    for (int i = 0; i < e.vl; ++i)
      for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t)
          for (int j = 0; j < e.vr; ++j)
            W[((size_t(oa + i) * d + s) * d + t) * w + (ob + j)] = e.at(i, s, t, j);
  }
}

}  // namespace

// Per-site construction for the finite chain; sites with byte-identical blocks
// share one construction. Output: W_i as host complex arrays [wl][d][d][wr] with
// the boundary rows/columns already selected (wl = 1 at site 0, wr = 1 at L-1).
int build_mpo_host(int L, int d, int chi, const double* A, const double* B, const double* C,
                   const double* Dh, int N, double tau_re, double tau_im, int variant,
                   std::vector<std::vector<std::complex<double>>>& sites, std::vector<int>& wl,
                   std::vector<int>& wr) {
  const cplx tau(tau_re, tau_im);
  const size_t nA = size_t(chi) * chi * d * d, nB = size_t(chi) * d * d, nD = size_t(d) * d;
  std::map<std::string, std::pair<std::vector<cplx>, int>> cache;
  sites.assign(L, {});
  wl.assign(L, 0);
  wr.assign(L, 0);
  for (int i = 0; i < L; ++i) {
    Blocks blk{chi, d, A + 2 * nA * i, B + 2 * nB * i, C + 2 * nB * i, Dh + 2 * nD * i};
    std::string key;
    key.append(reinterpret_cast<const char*>(blk.A), 16 * nA);
    key.append(reinterpret_cast<const char*>(blk.B), 16 * nB);
    key.append(reinterpret_cast<const char*>(blk.C), 16 * nB);
    key.append(reinterpret_cast<const char*>(blk.D), 16 * nD);
    auto it = cache.find(key);
    if (it == cache.end()) {
      std::vector<cplx> W;
      int w = 0;
      std::vector<int> offs;
      build_site(blk, N, tau, variant, W, w, offs);
      it = cache.emplace(key, std::make_pair(std::move(W), w)).first;
    }
    const std::vector<cplx>& W = it->second.first;
    const int w = it->second.second;
    const int l0 = (i == 0) ? 1 : w, r0 = (i == L - 1) ? 1 : w;
    std::vector<cplx> S(size_t(l0) * d * d * r0);
    for (int a = 0; a < l0; ++a)
      for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t)
          for (int b = 0; b < r0; ++b) S[((size_t(a) * d + s) * d + t) * r0 + b] = W[((size_t(a) * d + s) * d + t) * w + b];
    sites[i] = std::move(S);
    wl[i] = l0;
    wr[i] = r0;
  }
  return 0;
}

}  // namespace tevo
