// C-ABI entry points and the host-side plan of the compressed-Taylor FMM.
//
// The plan realises Sec. 3.1 of the paper without forming the dense matrices:
// with the last axis slowest (Lemma 5), row n of the PDE matrix P pivots on
// n + c e_s, so the decompression operator of eq. (decompression) is the
// sparse recurrence (Thm 4)
//     D[m] = sum_{xi != c e_s} (-a_xi / a_{c e_s}) D[m - c e_s + xi],  m_s >= c,
// swept slab by slab upward; its transpose (compression, eq.
// (define_beta_multipole)) is the same recurrence swept downward in gather form.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "adaptive.cuh"
#include "fmm_internal.cuh"

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Slab layout (see fmm_internal.cuh): row bases for order P with slabs 0..nslab-1.
struct Layout {
  int d = 0, P = 0, nslab = 0, n = 0;
  std::vector<int> row;
  int index(const int* m) const {  // m = (m0, m1, ms) for d=3, (m0, ms) for d=2
    if (d == 3) return row[(size_t)m[2] * (P + 1) + m[1]] + m[0];
    return row[(size_t)m[1]] + m[0];
  }
};

Layout make_layout(int d, int P, int nslab) {
  Layout L;
  L.d = d;
  L.P = P;
  L.nslab = nslab;
  int pos = 0;
  if (d == 3) {
    L.row.assign((size_t)(P + 1) * (P + 1), -1);
    for (int ms = 0; ms < nslab && ms <= P; ++ms)
      for (int m1 = 0; m1 <= P - ms; ++m1) {
        L.row[(size_t)ms * (P + 1) + m1] = pos;
        pos += P - ms - m1 + 1;
      }
  } else {
    L.row.assign((size_t)(P + 1), -1);
    for (int ms = 0; ms < nslab && ms <= P; ++ms) {
      L.row[ms] = pos;
      pos += P - ms + 1;
    }
  }
  L.n = pos;
  return L;
}

// Enumerate the full layout of order P (all slabs) into multi-indices.
std::vector<std::array<int, 3>> enumerate_full(int d, int P) {
  std::vector<std::array<int, 3>> out;
  if (d == 3) {
    for (int ms = 0; ms <= P; ++ms)
      for (int m1 = 0; m1 <= P - ms; ++m1)
        for (int m0 = 0; m0 <= P - ms - m1; ++m0) out.push_back({m0, m1, ms});
  } else {
    for (int ms = 0; ms <= P; ++ms)
      for (int m0 = 0; m0 <= P - ms; ++m0) out.push_back({m0, ms, 0});
  }
  return out;
}

using Key = std::array<int, 3>;

// The kernel's own PDE (eq. (define_pde_op)); multi-indices padded to 3.
std::map<Key, double> default_pde(int kernel, int d, double lam) {
  std::map<Key, double> a;
  auto e2 = [&](int k) {
    Key m{0, 0, 0};
    m[k] = 2;
    return m;
  };
  if (kernel == FMM_KERNEL_LAPLACE || kernel == FMM_KERNEL_YUKAWA ||
      kernel == FMM_KERNEL_HELMHOLTZ) {
    for (int k = 0; k < d; ++k) a[e2(k)] += 1.0;
    if (kernel == FMM_KERNEL_YUKAWA) a[Key{0, 0, 0}] += -lam * lam;
    if (kernel == FMM_KERNEL_HELMHOLTZ) a[Key{0, 0, 0}] += lam * lam;  // kappa = lam
  } else if (kernel == FMM_KERNEL_BIHARMONIC) {
    for (int k = 0; k < d; ++k)
      for (int l = 0; l < d; ++l) {
        Key m{0, 0, 0};
        m[k] += 2;
        m[l] += 2;
        a[m] += 1.0;
      }
  }
  return a;
}

template <typename T>
T* carve(char*& cur, size_t count) {
  T* p = reinterpret_cast<T*>(cur);
  cur += align_up(count * sizeof(T));
  return p;
}

int to_status(cudaError_t e) { return e == cudaSuccess ? FMM_OK : FMM_ERR_CUDA; }

}  // namespace

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
// adaptive plans (levels < 0, 3D, FP64): points, sort scratch, Morton codes,
// box arrays sized by the bound on the number of boxes, expansions per box
static int workspace_layout_adaptive(const fmm_plan_s* P, int64_t n_src, int64_t n_tgt,
                                     void* base, Workspace* ws) {
  const int D = -P->desc.levels, nj = P->pd.nj, nh = P->pd.nh;
  const int64_t nmax = std::max<int64_t>(std::max(n_src, n_tgt), 1);
  const int64_t nblk = (nmax + 1023) / 1024;
  const int64_t nb = adaptive_box_bound(n_src + n_tgt, P->desc.max_leaf, D);
  char* cur = static_cast<char*>(base);
  Workspace w{};
  w.geom = carve<Geom>(cur, 1);
  for (int k = 0; k < 3; ++k) w.sx[k] = carve<double>(cur, std::max<int64_t>(n_src, 1));
  w.sw = carve<double>(cur, std::max<int64_t>(n_src, 1));
  w.sperm = carve<int>(cur, std::max<int64_t>(n_src, 1));
  for (int k = 0; k < 3; ++k) w.tx[k] = carve<double>(cur, std::max<int64_t>(n_tgt, 1));
  w.tperm = carve<int>(cur, std::max<int64_t>(n_tgt, 1));
  w.keys_a = carve<uint32_t>(cur, nmax);
  w.keys_b = carve<uint32_t>(cur, nmax);
  w.vals_a = carve<int>(cur, nmax);
  w.vals_b = carve<int>(cur, nmax);
  w.skey = carve<uint32_t>(cur, std::max<int64_t>(n_src, 1));
  w.tkey = carve<uint32_t>(cur, std::max<int64_t>(n_tgt, 1));
  const int64_t nhist = 256 * nblk;
  const int64_t nscan = std::max<int64_t>(nhist, nb + 1);
  w.hist = carve<int>(cur, nhist);
  w.hist_sums = carve<int>(cur, (nscan + 1023) / 1024 + 1);
  w.anb_cap = nb;
  w.akey = carve<uint32_t>(cur, nb);
  w.alev = carve<int>(cur, nb);
  w.apar = carve<int>(cur, nb);
  w.achild = carve<int>(cur, 8 * nb);
  w.as0 = carve<int>(cur, nb);
  w.as1 = carve<int>(cur, nb);
  w.at0 = carve<int>(cur, nb);
  w.at1 = carve<int>(cur, nb);
  w.aleaf = carve<int>(cur, nb);
  w.am2p = carve<unsigned char>(cur, nb);
  if (P->desc.precision != FMM_PREC_FP64 && P->pd.d == 3) {
    w.asxh = carve<float4>(cur, std::max<int64_t>(n_src, 1));
    w.asxl = carve<float4>(cur, std::max<int64_t>(n_src, 1));
  }
  w.aloff = carve<int>(cur, FMM_MAX_ADEPTH + 4 + 6 * (FMM_MAX_ADEPTH + 2));
  w.anch = carve<int>(cur, nb);
  w.ascan = carve<int>(cur, nb + 1);
  w.mp = carve<double>(cur, (size_t)nb * nj);
  w.lc = carve<double>(cur, (size_t)nb * nj);
  w.agrid = carve<int>(cur, (size_t)agrid_offset(std::min(D, FMM_AGRID_LEVELS) + 1));
  w.htab = carve<double>(cur, (size_t)std::max(D - 1, 1) * 343 * nh);
  w.nbbox_blocks = (int)std::min<int64_t>(1024, (std::max(n_src, n_tgt) + 255) / 256 + 1);
  w.bbox = carve<double>(cur, (size_t)2 * 3 * 2 * w.nbbox_blocks);
  const int prec = P->desc.precision;
  if (prec_tensor(prec)) {
    const TcShape tcs = tc_shape(nj, prec);
    const int esz = tcs.esz;
    w.tc_jp = tcs.jp;
    w.tc_mp = tcs.npt;
    const int halves = prec == FMM_PREC_TF32 ? 1 : 2;
    const int tlev = kernel_homogeneous(P->pd.kernel) ? 1 : std::max(D - 1, 1);
    for (int h = 0; h < halves; ++h)
      w.tc_tmat[h] = carve<char>(cur, (size_t)tlev * 343 * w.tc_mp * w.tc_jp * esz);
    // window cells: as many as the bound on boxes (levels the arena cannot
    // hold fall back to the float CUDA-core M2L)
    w.tc_arena_bytes = (size_t)nb * ((size_t)w.tc_jp * esz * halves + sizeof(int));
    w.tc_arena = carve<char>(cur, w.tc_arena_bytes);
  }
  w.bytes = (size_t)(cur - static_cast<char*>(base));
  if (ws) *ws = w;
  return FMM_OK;
}

int fmm_workspace_layout(const fmm_plan_s* P, int64_t n_src, int64_t n_tgt, void* base,
                         Workspace* ws) {
  if (P->desc.levels < 0) return workspace_layout_adaptive(P, n_src, n_tgt, base, ws);
  const int d = P->pd.d, L = P->desc.levels, nj = P->pd.nj, nh = P->pd.nh;
  const int64_t nleaf = nbox_at(d, L);
  const int64_t nmax = std::max<int64_t>(std::max(n_src, n_tgt), 1);
  const int64_t nblk = (nmax + 1023) / 1024;
  char* cur = static_cast<char*>(base);
  Workspace w{};
  w.geom = carve<Geom>(cur, 1);
  for (int k = 0; k < d; ++k) w.sx[k] = carve<double>(cur, std::max<int64_t>(n_src, 1));
  w.sw = carve<double>(cur, std::max<int64_t>(n_src, 1));
  w.sperm = carve<int>(cur, std::max<int64_t>(n_src, 1));
  for (int k = 0; k < d; ++k) w.tx[k] = carve<double>(cur, std::max<int64_t>(n_tgt, 1));
  w.tperm = carve<int>(cur, std::max<int64_t>(n_tgt, 1));
  w.sstart = carve<int>(cur, nleaf + 1);
  w.tstart = carve<int>(cur, nleaf + 1);
  w.counts = carve<int>(cur, nleaf);
  w.keys_a = carve<uint32_t>(cur, nmax);
  w.keys_b = carve<uint32_t>(cur, nmax);
  w.vals_a = carve<int>(cur, nmax);
  w.vals_b = carve<int>(cur, nmax);
  const int64_t nhist = 256 * nblk;
  const int64_t nscan = std::max<int64_t>(nhist, nleaf + 1);
  w.hist = carve<int>(cur, nscan);
  w.hist_sums = carve<int>(cur, (nscan + 1023) / 1024 + 1);
  int64_t off = 0;
  for (int l = 0; l <= L; ++l) {
    w.lev_off[l] = off;
    if (l >= 2) off += nbox_at(d, l);
  }
  w.lev_off[L + 1] = off;
  w.mp = carve<double>(cur, (size_t)off * nj);
  w.lc = carve<double>(cur, (size_t)off * nj);
  const int noff = d == 3 ? 343 : 49;
  w.htab = carve<double>(cur, (size_t)(L - 1) * noff * nh);
  w.nbbox_blocks = (int)std::min<int64_t>(1024, (std::max(n_src, n_tgt) + 255) / 256 + 1);
  w.bbox = carve<double>(cur, (size_t)2 * 3 * 2 * w.nbbox_blocks);
  const int prec = P->desc.precision;
  if (d == 3 && prec != FMM_PREC_FP64) {
    w.sxr = carve<float4>(cur, std::max<int64_t>(n_src, 1));
    w.txr = carve<float4>(cur, std::max<int64_t>(n_tgt, 1));
  }
  if (d == 3 && prec_tensor(prec)) {
    const TcShape tcs = tc_shape(nj, prec);
    const int esz = tcs.esz;  // bytes per operand element
    w.tc_jp = tcs.jp;
    w.tc_mp = tcs.npt;
    const int halves = prec == FMM_PREC_TF32 ? 1 : 2;
    // homogeneous kernels (3D Laplace, biharmonic) share one set of offset
    // matrices across levels (exact power-of-two scale per level)
    const int tlev = kernel_homogeneous(P->pd.kernel) ? 1 : (L - 1);
    for (int h = 0; h < halves; ++h) {
      w.tc_bpar[h] = carve<char>(cur, (size_t)off * w.tc_jp * esz);
      w.tc_tmat[h] = carve<char>(cur, (size_t)tlev * 343 * w.tc_mp * w.tc_jp * esz);
    }
    if (prec == FMM_PREC_F16X3) w.tc_bscale = carve<float>(cur, (size_t)off);
  }
  if (P->pd.kernel == FMM_KERNEL_HELMHOLTZ) {
    // the real and imaginary parts' potentials (and gradients) before they are
    // interleaved into the caller's complex output
    w.hphi = carve<double>(cur, (size_t)2 * std::max<int64_t>(n_tgt, 1));
    w.hgrad = carve<double>(cur, (size_t)2 * d * std::max<int64_t>(n_tgt, 1));
  }
  if (P->desc.m2l == FMM_M2L_FFT) {
    const size_t csz = prec == FMM_PREC_FP64 ? 16 : 8;  // complex double / float
    const int tl = m2l_shared_tables(P) ? 1 : L - 1;
    w.fft_b = carve<char>(cur, (size_t)off * P->fft.kfp * csz);
    w.fft_g = carve<char>(cur, (size_t)off * P->fft.kfp * csz);
    w.fft_h = carve<char>(cur, (size_t)tl * noff * P->fft.kfp * csz);
  }
  w.bytes = (size_t)(cur - static_cast<char*>(base));
  if (ws) *ws = w;
  return FMM_OK;
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
// residual of a PDE on the kernel's derivatives (expansions.cu)
double pde_residual(const PlanDev& pd, const std::vector<int>& hrow_host, int nterm,
                    const int* xi, const double* a);

extern "C" int fmm_plan_create(fmm_plan_t* out, const fmm_plan_desc* desc) {
  if (!out) return FMM_ERR_ARG;
  *out = nullptr;
  if (!desc) return FMM_ERR_ARG;
  const int d = desc->d, p = desc->p, L = desc->levels;
  if (d != 2 && d != 3) return FMM_ERR_ARG;
  if (p < 1 || p > FMM_MAXP) return FMM_ERR_ARG;
  if (L < 0) {  // adaptive tree
    if (-L > FMM_MAX_ADEPTH || desc->max_leaf < 1) return FMM_ERR_ARG;
    if (d != 3 || desc->m2l == FMM_M2L_FFT) return FMM_ERR_UNSUPPORTED;
  } else if (L < 2 || L > (d == 3 ? 7 : 8)) {
    return FMM_ERR_ARG;
  }
  if (desc->precision < FMM_PREC_FP64 || desc->precision > FMM_PREC_F16X3) return FMM_ERR_ARG;
  // the F16X3 scalings are laid out for the uniform trees' parent grids
  if (desc->precision == FMM_PREC_F16X3 && desc->levels < 0) return FMM_ERR_UNSUPPORTED;
  if (desc->m2l != FMM_M2L_DENSE && desc->m2l != FMM_M2L_FFT && desc->m2l != FMM_M2L_AUTO)
    return FMM_ERR_ARG;
  if (desc->m2l == FMM_M2L_FFT && desc->precision != FMM_PREC_FP64 &&
      desc->precision != FMM_PREC_FP32)
    return FMM_ERR_UNSUPPORTED;
  const int kernel = desc->kernel;
  if (kernel == FMM_KERNEL_LAPLACE || kernel == FMM_KERNEL_BIHARMONIC) {
  } else if (kernel == FMM_KERNEL_YUKAWA || kernel == FMM_KERNEL_HELMHOLTZ) {
    if (d != 3) return FMM_ERR_UNSUPPORTED;
  } else {
    return FMM_ERR_ARG;
  }
  if ((kernel == FMM_KERNEL_YUKAWA || kernel == FMM_KERNEL_HELMHOLTZ) && !(desc->lambda > 0.0))
    return FMM_ERR_ARG;
  if (kernel == FMM_KERNEL_HELMHOLTZ && L < 0) return FMM_ERR_UNSUPPORTED;  // uniform trees
  for (int k = 0; k < d; ++k)
    if (!std::isfinite(desc->root_lo[k])) return FMM_ERR_ARG;

  // PDE coefficients
  std::map<Key, double> a;
  if (desc->pde) {
    if (desc->pde->n_terms <= 0 || !desc->pde->multi_idx || !desc->pde->coeff) return FMM_ERR_ARG;
    for (int t = 0; t < desc->pde->n_terms; ++t) {
      Key m{0, 0, 0};
      for (int k = 0; k < d; ++k) {
        m[k] = desc->pde->multi_idx[t * d + k];
        if (m[k] < 0) return FMM_ERR_ARG;
      }
      a[m] += desc->pde->coeff[t];
    }
  } else {
    a = default_pde(kernel, d, desc->lambda);
  }
  int c = 0;
  for (auto& kv : a)
    if (kv.second != 0.0) c = std::max(c, kv.first[0] + kv.first[1] + kv.first[2]);
  if (c < 1) return FMM_ERR_UNSUPPORTED;
  Key lead{0, 0, 0};
  lead[d - 1] = c;
  const double alead = a.count(lead) ? a[lead] : 0.0;
  if (alead == 0.0) return FMM_ERR_UNSUPPORTED;  // Property 1 on the last axis

  PlanDev pd{};
  pd.d = d;
  pd.p = p;
  pd.c = c;
  pd.kernel = kernel;
  pd.lam = desc->lambda;
  for (auto& kv : a) {
    if (kv.second == 0.0 || kv.first == lead) continue;
    if (pd.nterms >= FMM_MAX_TERMS) return FMM_ERR_UNSUPPORTED;
    int t = pd.nterms++;
    int deg = 0;
    for (int k = 0; k < 3; ++k) {
      pd.tsh[t][k] = kv.first[k] - lead[k];
      deg += kv.first[k];
    }
    pd.tcoef[t] = -kv.second / alead;
    pd.tcoef_f[t] = (float)pd.tcoef[t];
    pd.tpow[t] = c - deg;
  }

  Layout full = make_layout(d, p, p + 1);
  Layout hank = make_layout(d, 2 * p, 2 * c - 1);
  pd.nfull = full.n;
  pd.nh = hank.n;
  {
    Key m{0, 0, 0};
    m[d - 1] = std::min(c, p + 1);
    pd.nj = (c > p) ? full.n : (d == 3 ? full.row[(size_t)c * (p + 1)] : full.row[c]);
  }
  auto mis = enumerate_full(d, p);
  if ((int)mis.size() != pd.nfull) return FMM_ERR_UNSUPPORTED;

  // host tables
  std::vector<char4> mi(pd.nfull);
  std::vector<double> inv_fact(pd.nfull);
  const int nt = std::max(pd.nterms, 1);
  std::vector<int16_t> rec(pd.nfull * (size_t)nt, -1), cmp(pd.nfull * (size_t)nt, -1);
  for (int i = 0; i < pd.nfull; ++i) {
    const auto& m = mis[i];
    const int ms = m[d - 1];
    const int deg = m[0] + m[1] + m[2];
    mi[i] = make_char4((char)m[0], (char)m[1], (char)m[2], (char)deg);
    double f = 1.0;
    for (int k = 0; k < 3; ++k)
      for (int t = 2; t <= m[k]; ++t) f *= t;
    inv_fact[i] = 1.0 / f;
    if (full.index(m.data()) != i) return FMM_ERR_UNSUPPORTED;
    for (int t = 0; t < pd.nterms; ++t) {
      // decompression source m + shift (rows with m_s >= c)
      if (ms >= c) {
        int q[3];
        for (int k = 0; k < 3; ++k) q[k] = m[k] + pd.tsh[t][k];
        rec[(size_t)i * nt + t] = (int16_t)full.index(q);
      }
      // compression gather source m - shift (must be in M(p) with m_s >= c)
      int q[3], ok = 1, qd = 0;
      for (int k = 0; k < 3; ++k) {
        q[k] = m[k] - pd.tsh[t][k];
        if (q[k] < 0) ok = 0;
        qd += q[k];
      }
      if (ok && qd <= p && q[d - 1] >= c) cmp[(size_t)i * nt + t] = (int16_t)full.index(q);
    }
  }

  // upload
  const size_t n_mi = align_up(sizeof(char4) * pd.nfull);
  const size_t n_if = align_up(sizeof(double) * pd.nfull);
  const size_t n_iff = align_up(sizeof(float) * pd.nfull);
  const size_t n_rc = align_up(sizeof(int16_t) * pd.nfull * nt);
  const size_t n_fr = align_up(sizeof(int) * full.row.size());
  const size_t n_hr = align_up(sizeof(int) * hank.row.size());
  // FFT form of M2L: transform lengths, twiddles and the scaling g^{+-n}
  FftDev fft{};
  fft.n1 = 2 * p + 1;
  fft.n2 = d == 3 ? 2 * p + 1 : 1;
  fft.n3 = 2 * std::min(c, p + 1) - 1;  // M_s = max m_s over j
  fft.k1 = p + 1;
  fft.kf = fft.k1 * fft.n2 * fft.n3;
  fft.kfp = (fft.kf + 31) / 32 * 32;
  std::vector<double> ftab;
  const double kPi = 3.14159265358979323846;
  for (int n = 0; n < fft.n1; ++n) {
    ftab.push_back(std::cos(2.0 * kPi * n / fft.n1));
    ftab.push_back(std::sin(2.0 * kPi * n / fft.n1));
  }
  for (int n = 0; n < fft.n3; ++n) {
    ftab.push_back(std::cos(2.0 * kPi * n / fft.n3));
    ftab.push_back(std::sin(2.0 * kPi * n / fft.n3));
  }
  // scaling of Sec. 4.1.1 in units of the box side: g = 3p/8 (at least 1)
  // balances the magnitudes of the scaled multipoles and derivatives
  const double g = std::max(1.0, 0.375 * p);
  for (int n = 0; n <= 2 * p; ++n) ftab.push_back(std::pow(g, n));
  for (int n = 0; n <= 2 * p; ++n) ftab.push_back(std::pow(g, -n));
  const size_t n_ft = align_up(sizeof(double) * ftab.size());
  // P2M monomial segments (d = 3): each row (m_1, m_s) of the full layout cut
  // into runs of at most 4 consecutive m_0
  std::vector<int> seg;
  if (d == 3)
    for (int ms = 0; ms <= p; ++ms)
      for (int m1 = 0; m1 <= p - ms; ++m1) {
        const int len = p - ms - m1 + 1;
        for (int a = 0; a < len; a += 4) {
          const int pos = full.row[(size_t)ms * (p + 1) + m1] + a;
          seg.push_back(a | (m1 << 5) | (ms << 10) | (std::min(4, len - a) << 15) | (pos << 18));
        }
      }
  pd.p2m_nseg = (int)seg.size();
  const size_t n_sg = align_up(sizeof(int) * std::max<size_t>(seg.size(), 1));
  const size_t total = n_mi + n_if + 2 * n_rc + n_fr + n_hr + n_ft + 2 * n_iff + n_sg;
  std::vector<char> host(total, 0);
  char* h = host.data();
  {
    std::vector<float> iff(pd.nfull), ff(pd.nfull);
    for (int i = 0; i < pd.nfull; ++i) {
      iff[i] = (float)inv_fact[i];
      // m! (sqrt 2)^|m| (m! < 2^53: exact in double): the F16X3 operand scale
      ff[i] = (float)(1.0 / inv_fact[i] * std::pow(std::sqrt(2.0), (double)mi[i].w));
    }
    std::memcpy(h + total - n_sg - 2 * n_iff, iff.data(), sizeof(float) * pd.nfull);
    std::memcpy(h + total - n_sg - n_iff, ff.data(), sizeof(float) * pd.nfull);
  }
  if (!seg.empty()) std::memcpy(h + total - n_sg, seg.data(), sizeof(int) * seg.size());
  std::memcpy(h, mi.data(), sizeof(char4) * pd.nfull);
  std::memcpy(h + n_mi, inv_fact.data(), sizeof(double) * pd.nfull);
  std::memcpy(h + n_mi + n_if, rec.data(), sizeof(int16_t) * rec.size());
  std::memcpy(h + n_mi + n_if + n_rc, cmp.data(), sizeof(int16_t) * cmp.size());
  std::memcpy(h + n_mi + n_if + 2 * n_rc, full.row.data(), sizeof(int) * full.row.size());
  std::memcpy(h + n_mi + n_if + 2 * n_rc + n_fr, hank.row.data(), sizeof(int) * hank.row.size());
  std::memcpy(h + n_mi + n_if + 2 * n_rc + n_fr + n_hr, ftab.data(), sizeof(double) * ftab.size());
  void* dt = nullptr;
  if (cudaMalloc(&dt, total) != cudaSuccess) return FMM_ERR_NOMEM;
  if (cudaMemcpy(dt, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dt);
    return FMM_ERR_CUDA;
  }
  char* db = static_cast<char*>(dt);
  pd.mi = reinterpret_cast<const char4*>(db);
  pd.inv_fact = reinterpret_cast<const double*>(db + n_mi);
  pd.inv_fact_f = reinterpret_cast<const float*>(db + total - n_sg - 2 * n_iff);
  pd.fact_f = reinterpret_cast<const float*>(db + total - n_sg - n_iff);
  pd.p2m_seg = reinterpret_cast<const int*>(db + total - n_sg);
  pd.rec_src = reinterpret_cast<const int16_t*>(db + n_mi + n_if);
  pd.cmp_src = reinterpret_cast<const int16_t*>(db + n_mi + n_if + n_rc);
  pd.frow = reinterpret_cast<const int*>(db + n_mi + n_if + 2 * n_rc);
  pd.hrow = reinterpret_cast<const int*>(db + n_mi + n_if + 2 * n_rc + n_fr);
  {
    const double* ft = reinterpret_cast<const double*>(db + n_mi + n_if + 2 * n_rc + n_fr + n_hr);
    fft.tw1 = ft;
    fft.tw3 = ft + 2 * fft.n1;
    fft.gpow = ft + 2 * fft.n1 + 2 * fft.n3;
  }

  fmm_plan_s* P = new (std::nothrow) fmm_plan_s();
  if (!P) {
    cudaFree(dt);
    return FMM_ERR_NOMEM;
  }
  {  // the plan's two streams and their events; on failure release what was made
    int prio_low = 0, prio_high = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&P->hi, cudaStreamNonBlocking, prio_high) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&P->aux, cudaStreamNonBlocking, prio_low) == cudaSuccess;
    cudaEvent_t* evs[5] = {&P->ev_in, &P->ev_fork, &P->ev_join, &P->ev_out, &P->ev_tab};
    for (cudaEvent_t* e : evs)
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      for (cudaEvent_t* e : evs)
        if (*e) cudaEventDestroy(*e);
      if (P->aux) cudaStreamDestroy(P->aux);
      if (P->hi) cudaStreamDestroy(P->hi);
      cudaFree(dt);
      delete P;
      return FMM_ERR_CUDA;
    }
  }
  if (desc->pde && c >= 2 && c <= p) {
    // a user PDE must be satisfied by the kernel, or the compression of Sec. 3
    // would discard information the potential needs (eq. (Pv))
    std::vector<int> xi;
    std::vector<double> av;
    for (auto& kv : a) {
      if (kv.second == 0.0) continue;
      xi.insert(xi.end(), {kv.first[0], kv.first[1], kv.first[2]});
      av.push_back(kv.second);
    }
    const int kinds = kernel == FMM_KERNEL_HELMHOLTZ ? 2 : 1;
    for (int part = 0; part < kinds; ++part) {
      PlanDev q = pd;
      if (part == 1) q.kernel = kHelmIm;
      const double res = pde_residual(q, hank.row, (int)av.size(), xi.data(), av.data());
      if (res < 0.0 || res > 1e-10) {
        cudaStreamDestroy(P->hi);
        cudaStreamDestroy(P->aux);
        for (cudaEvent_t e : {P->ev_in, P->ev_fork, P->ev_join, P->ev_out, P->ev_tab})
          cudaEventDestroy(e);
        cudaFree(dt);
        delete P;
        return res < 0.0 ? FMM_ERR_CUDA : FMM_ERR_UNSUPPORTED;
      }
    }
  }
  P->desc = *desc;
  P->desc.pde = nullptr;
  if (desc->m2l == FMM_M2L_AUTO) {  // resolved once, by arithmetic (see ctfmm.h)
    const bool fp = desc->precision == FMM_PREC_FP64 || desc->precision == FMM_PREC_FP32;
    P->desc.m2l = (fp && desc->levels > 0) ? FMM_M2L_FFT : FMM_M2L_DENSE;
  }
  P->pd = pd;
  P->fft = fft;
  P->dev_tables = dt;
  *out = P;
  return FMM_OK;
}

extern "C" int fmm_plan_destroy(fmm_plan_t P) {
  if (!P) return FMM_ERR_ARG;
  cudaDeviceSynchronize();
  if (P->events_made)
    for (auto& e : P->ev) cudaEventDestroy(e);
  if (P->events_made)
    for (auto& e : P->evk) cudaEventDestroy(e);
  for (cudaEvent_t e : {P->ev_in, P->ev_fork, P->ev_join, P->ev_out, P->ev_tab})
    cudaEventDestroy(e);
  cudaStreamDestroy(P->hi);
  cudaStreamDestroy(P->aux);
  cudaFree(P->dev_tables);
  delete P;
  return FMM_OK;
}

extern "C" int fmm_plan_info(fmm_plan_t P, int* nfull, int* nj, int* c) {
  if (!P) return FMM_ERR_ARG;
  if (nfull) *nfull = P->pd.nfull;
  if (nj) *nj = P->pd.nj;
  if (c) *c = P->pd.c;
  return FMM_OK;
}

extern "C" int fmm_workspace_size(fmm_plan_t P, int64_t n_src, int64_t n_tgt, size_t* bytes) {
  if (!P || !bytes || n_src < 0 || n_tgt < 0) return FMM_ERR_ARG;
  if (n_src > INT32_MAX / 2 || n_tgt > INT32_MAX / 2) return FMM_ERR_ARG;
  Workspace w;
  fmm_workspace_layout(P, n_src, n_tgt, nullptr, &w);
  *bytes = w.bytes + kAlign;
  return FMM_OK;
}

extern "C" int fmm_set_timing(fmm_plan_t P, int enable) {
  if (!P) return FMM_ERR_ARG;
  if (enable && !P->events_made) {
    for (auto& e : P->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return FMM_ERR_CUDA;
    for (auto& e : P->evk)
      if (cudaEventCreate(&e) != cudaSuccess) return FMM_ERR_CUDA;
    P->events_made = true;
  }
  P->timing = enable ? 1 : 0;
  return FMM_OK;
}

extern "C" int fmm_phase_times(fmm_plan_t P, float* ms) {
  if (!P || !ms || !P->events_made) return FMM_ERR_ARG;
  if (cudaEventSynchronize(P->ev[FMM_NUM_PHASES]) != cudaSuccess) return FMM_ERR_CUDA;
  for (int i = 0; i < FMM_NUM_PHASES; ++i)
    if (cudaEventElapsedTime(&ms[i], P->ev[i], P->ev[i + 1]) != cudaSuccess) return FMM_ERR_CUDA;
  return FMM_OK;
}

extern "C" int fmm_m2l_kernel_time(fmm_plan_t P, float* ms) {
  if (!P || !ms || !P->events_made) return FMM_ERR_ARG;
  if (cudaEventSynchronize(P->evk[1]) != cudaSuccess) return FMM_ERR_CUDA;
  if (cudaEventElapsedTime(ms, P->evk[0], P->evk[1]) != cudaSuccess) return FMM_ERR_CUDA;
  return FMM_OK;
}

// M2L translations of a uniform tree: per level, the (target, source) pairs
// whose parents are adjacent minus those that are adjacent themselves; the
// count factorises over the axes.
static int64_t uniform_m2l_count(int d, int L) {
  int64_t tot = 0;
  for (int l = 2; l <= L; ++l) {
    const int64_t n = (int64_t)1 << l;
    int64_t A = 0, B = 0;
    for (int64_t t = 0; t < n; ++t)
      for (int64_t s = std::max<int64_t>(0, t - 3); s <= std::min<int64_t>(n - 1, t + 3); ++s) {
        const int64_t dp = (t >> 1) - (s >> 1);
        if (dp < -1 || dp > 1) continue;
        ++A;
        if (t - s >= -1 && t - s <= 1) ++B;
      }
    int64_t Ad = 1, Bd = 1;
    for (int k = 0; k < d; ++k) {
      Ad *= A;
      Bd *= B;
    }
    tot += Ad - Bd;
  }
  return tot;
}

extern "C" int fmm_last_tree(fmm_plan_t P, int64_t* boxes, int* depth, int64_t* m2l) {
  if (!P) return FMM_ERR_ARG;
  const int L = P->desc.levels;
  int64_t nb = 0;
  if (L > 0)
    for (int l = 0; l <= L; ++l) nb += nbox_at(P->pd.d, l);
  if (boxes) *boxes = L > 0 ? nb : P->last_boxes;
  if (depth) *depth = L > 0 ? L : P->last_depth;
  if (m2l) {
    if (L > 0) {
      *m2l = uniform_m2l_count(P->pd.d, L);
    } else {
      *m2l = 0;
      if (P->last_geom) {
        Geom g;
        if (cudaStreamSynchronize(P->last_stream) != cudaSuccess) return FMM_ERR_CUDA;
        if (cudaMemcpy(&g, P->last_geom, sizeof(Geom), cudaMemcpyDeviceToHost) != cudaSuccess)
          return FMM_ERR_CUDA;
        *m2l = (int64_t)g.m2l_count;
      }
    }
  }
  return FMM_OK;
}

extern "C" int fmm_last_launch_count(fmm_plan_t P) { return P ? P->launches : -1; }

// near-field pairs of a uniform tree: per target leaf, its targets times the
// sources of the 3^d leaves around it (the leaf included)
template <int D>
__global__ void k_count_pairs(int L, const int* __restrict__ sstart, const int* __restrict__ tstart,
                              unsigned long long* out) {
  const int64_t nl = (int64_t)1 << L, nleaf = (int64_t)1 << (D * L);
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (b < nleaf) {
    const int64_t x = b % nl, y = D == 3 ? (b / nl) % nl : b / nl, z = D == 3 ? b / (nl * nl) : 0;
    int64_t ns = 0;
    for (int64_t dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dx = -1; dx <= 1; ++dx) {
          const int64_t X = x + dx, Y = y + dy, Z = z + dz;
          if (X < 0 || Y < 0 || Z < 0 || X >= nl || Y >= nl || Z >= nl) continue;
          const int64_t n = (Z * nl + Y) * nl + X;
          ns += sstart[n + 1] - sstart[n];
        }
    v = (unsigned long long)(tstart[b + 1] - tstart[b]) * (unsigned long long)ns;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

extern "C" int fmm_last_stats(fmm_plan_t P, fmm_stats* out) {
  if (!P || !out) return FMM_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->p2p_pairs = -1;
  if (P->timing && P->events_made && P->last_geom) {
    if (fmm_phase_times(P, out->phase_ms) != FMM_OK) return FMM_ERR_CUDA;
    if (fmm_m2l_kernel_time(P, &out->m2l_kernel_ms) != FMM_OK) out->m2l_kernel_ms = 0.f;
  }
  int rc = fmm_last_tree(P, &out->boxes, &out->depth, &out->m2l_translations);
  if (rc != FMM_OK) return rc;
  out->status = fmm_last_status(P);
  out->launches = P->launches;
  if (P->timing && P->last_geom && P->desc.levels > 0 && P->pd.kernel != FMM_KERNEL_HELMHOLTZ) {
    Geom g;
    if (cudaMemcpy(&g, P->last_geom, sizeof(Geom), cudaMemcpyDeviceToHost) != cudaSuccess)
      return FMM_ERR_CUDA;
    out->p2p_pairs = (int64_t)g.p2p_pairs;
  }
  return FMM_OK;
}

extern "C" int fmm_set_wait_limit(fmm_plan_t P, long long cycles) {
  if (!P || cycles < 0) return FMM_ERR_ARG;
  P->tc_wait_cycles = cycles;
  return FMM_OK;
}

// ---------------------------------------------------------------------------
// Evaluation
// ---------------------------------------------------------------------------
// interleave the real and imaginary parts' results into complex output
__global__ void k_interleave(int64_t n, const double* __restrict__ re,
                             const double* __restrict__ im, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    out[2 * i] = re[i];
    out[2 * i + 1] = im[i];
  }
}

// Helmholtz (G = e^{i kappa r}/r): real weights give real multipoles, and the
// PDE Laplacian + kappa^2 has real coefficients, so the tree, P2M and M2M are
// shared; the derivative tables, M2L, L2L and the leaf pass run once with the
// real part cos(kappa r)/r and once with the imaginary part sin(kappa r)/r
// (every stage after M2M is linear in G).  One stream; phases 4..6 of the
// timing hold both parts.
static int eval_helmholtz(fmm_plan_t P, const Workspace& ws, int64_t n_src, const double* src,
                          const double* w, int64_t n_tgt, const double* tgt, double* phi,
                          double* grad, cudaStream_t st, bool first) {
  int nl = 0;
  auto mark = [&](int i) {
    if (P->timing) cudaEventRecord(P->ev[i], st);
  };
  mark(0);
  if (launch_set_geom(P, ws, n_src, src, n_tgt, tgt, st, &nl) != cudaSuccess) return FMM_ERR_CUDA;
  if (launch_build_tree(P, ws, n_src, src, w, n_tgt, tgt, st, &nl) != cudaSuccess)
    return FMM_ERR_CUDA;
  mark(1);
  mark(2);
  if (launch_p2m(P, ws, st, &nl) != cudaSuccess) return FMM_ERR_CUDA;
  mark(3);
  if (launch_m2m(P, ws, st, &nl) != cudaSuccess) return FMM_ERR_CUDA;
  mark(4);
  const int d = P->pd.d;
  for (int part = 0; part < 2; ++part) {
    fmm_plan_s Q = *P;
    Q.pd.kernel = part == 0 ? FMM_KERNEL_HELMHOLTZ : kHelmIm;
    double* ph = n_tgt > 0 ? ws.hphi + part * n_tgt : nullptr;
    double* gr = grad ? ws.hgrad + (size_t)part * d * n_tgt : nullptr;
    if (launch_deriv_tables(&Q, ws, st, &nl) != cudaSuccess) return FMM_ERR_CUDA;
    if (launch_m2l(&Q, ws, st, &nl, false) != cudaSuccess) return FMM_ERR_CUDA;
    if (launch_l2l(&Q, ws, st, &nl) != cudaSuccess) return FMM_ERR_CUDA;
    if (n_tgt > 0 && launch_leaf_eval(&Q, ws, ph, gr, st, &nl) != cudaSuccess)
      return FMM_ERR_CUDA;
  }
  mark(5);
  mark(6);
  if (n_tgt > 0) {
    k_interleave<<<(unsigned)((n_tgt + 255) / 256), 256, 0, st>>>(n_tgt, ws.hphi,
                                                                  ws.hphi + n_tgt, phi);
    ++nl;
    if (grad) {
      const int64_t ng = n_tgt * d;
      k_interleave<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(ng, ws.hgrad, ws.hgrad + ng,
                                                                 grad);
      ++nl;
    }
  }
  mark(7);
  if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
  P->last_stream = st;
  P->last_geom = ws.geom;
  P->launches = first ? nl : P->launches + nl;
  return FMM_OK;
}

static int eval_internal(fmm_plan_t P, int64_t n_src, const double* src, const double* w,
                         int64_t n_tgt, const double* tgt, double* phi, double* grad,
                         void* workspace, size_t wbytes, cudaStream_t st, bool first) {
  if (!P || n_src < 0 || n_tgt < 0) return FMM_ERR_ARG;
  if (n_src > 0 && (!src || !w)) return FMM_ERR_ARG;
  if (n_tgt > 0 && !tgt) return FMM_ERR_ARG;
  if (!workspace) return FMM_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return FMM_ERR_ARG;
  Workspace ws;
  fmm_workspace_layout(P, n_src, n_tgt, workspace, &ws);
  if (ws.bytes > wbytes) return FMM_ERR_WORKSPACE;
  if (tgt == src && n_tgt == n_src) {
    // targets are the sources: one sort serves both (same keys, same stable order)
    for (int k = 0; k < 3; ++k) ws.tx[k] = ws.sx[k];
    ws.tperm = ws.sperm;
    ws.tstart = ws.sstart;
    ws.txr = ws.sxr;
    ws.tkey = ws.skey;
  }
  int nl = 0;
  cudaError_t e = cudaSuccess;
  // FP32 3D uniform path: the near field needs only the sorted points, so it
  // runs on a low-priority stream of the plan while the rest of the pipeline
  // runs on a high-priority one (the block scheduler then fills the SMs the
  // memory-bound passes and the tensor-core M2L leave idle with near-field
  // blocks); both are ordered after the caller's stream and the caller's
  // stream after both
  const bool split = P->desc.levels > 0 && leaf_split_supported(P) && n_tgt > 0;
  cudaStream_t run = split ? P->hi : st;
  auto mark = [&](int i) {
    if (P->timing) cudaEventRecord(P->ev[i], run);
  };
  if (P->desc.levels < 0) {
    if (grad) return FMM_ERR_UNSUPPORTED;
    {  // the adaptive build reads the level sizes back to the host once: not capturable
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FMM_ERR_CUDA;
      if (cs != cudaStreamCaptureStatusNone) return FMM_ERR_UNSUPPORTED;
    }
    mark(0);
    if ((e = launch_set_geom(P, ws, n_src, src, n_tgt, tgt, st, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    ATree tree;
    int overflow = 0;
    if ((e = launch_build_adaptive(P, ws, n_src, src, w, n_tgt, tgt, st, &nl, &tree, &overflow)) !=
        cudaSuccess)
      return FMM_ERR_CUDA;
    if (overflow) return FMM_ERR_WORKSPACE;
    const int nbox = tree.loff[tree.maxlev + 1];
    cudaMemsetAsync(ws.mp, 0, sizeof(double) * (size_t)nbox * P->pd.nj, st);
    cudaMemsetAsync(ws.lc, 0, sizeof(double) * (size_t)nbox * P->pd.nj, st);
    mark(1);
    if (tree.maxlev >= 2) {
      set_deriv_levels(P, tree.maxlev);
      if ((e = launch_deriv_tables(P, ws, st, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    }
    mark(2);
    if ((e = launch_adaptive_upward(P, ws, tree, st, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    mark(3);
    mark(4);
    if ((e = launch_adaptive_m2l(P, ws, tree, st, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    mark(5);
    if ((e = launch_adaptive_p2l_l2l(P, ws, tree, st, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    mark(6);
    if (n_tgt > 0 && (e = launch_adaptive_leaf(P, ws, tree, phi, st, &nl)) != cudaSuccess)
      return FMM_ERR_CUDA;
    mark(7);
    P->last_stream = st;
    P->last_geom = ws.geom;
    P->launches = first ? nl : P->launches + nl;
    P->last_boxes = nbox;
    P->last_depth = tree.maxlev;
    return FMM_OK;
  }
  if (P->pd.kernel == FMM_KERNEL_HELMHOLTZ)
    return eval_helmholtz(P, ws, n_src, src, w, n_tgt, tgt, phi, grad, st, first);
  if (split && (cudaEventRecord(P->ev_in, st) != cudaSuccess ||
                cudaStreamWaitEvent(run, P->ev_in, 0) != cudaSuccess))
    return FMM_ERR_CUDA;
  mark(0);
  if ((e = launch_set_geom(P, ws, n_src, src, n_tgt, tgt, run, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
  if ((e = launch_build_tree(P, ws, n_src, src, w, n_tgt, tgt, run, &nl)) != cudaSuccess)
    return FMM_ERR_CUDA;
  if (split) {
    // the derivative and offset tables depend only on the geometry: they are
    // built on the side stream while P2M and M2M run, then the near field
    if (cudaEventRecord(P->ev_fork, run) != cudaSuccess ||
        cudaStreamWaitEvent(P->aux, P->ev_fork, 0) != cudaSuccess)
      return FMM_ERR_CUDA;
    if ((e = launch_deriv_tables(P, ws, P->aux, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    if ((e = launch_m2l_tables(P, ws, P->aux, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    if (cudaEventRecord(P->ev_tab, P->aux) != cudaSuccess) return FMM_ERR_CUDA;
    if ((e = launch_near_field(P, ws, phi, grad, P->aux, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
    if (cudaEventRecord(P->ev_join, P->aux) != cudaSuccess) return FMM_ERR_CUDA;
  }
  mark(1);
  if (!split && (e = launch_deriv_tables(P, ws, run, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
  mark(2);
  if ((e = launch_p2m(P, ws, run, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
  mark(3);
  if ((e = launch_m2m(P, ws, run, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
  mark(4);
  if (split && cudaStreamWaitEvent(run, P->ev_tab, 0) != cudaSuccess) return FMM_ERR_CUDA;
  if ((e = launch_m2l(P, ws, run, &nl, split)) != cudaSuccess) return FMM_ERR_CUDA;
  mark(5);
  if ((e = launch_l2l(P, ws, run, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
  mark(6);
  if (split) {
    if (cudaStreamWaitEvent(run, P->ev_join, 0) != cudaSuccess) return FMM_ERR_CUDA;
    if ((e = launch_far_field(P, ws, phi, grad, run, &nl)) != cudaSuccess) return FMM_ERR_CUDA;
  } else if ((e = launch_leaf_eval(P, ws, phi, grad, run, &nl)) != cudaSuccess) {
    return FMM_ERR_CUDA;
  }
  mark(7);
  if (P->timing) {  // statistics: near-field pairs, after the timed phases
    const int64_t nleaf = nbox_at(P->pd.d, P->desc.levels);
    const unsigned nbk = (unsigned)((nleaf + 255) / 256);
    if (P->pd.d == 3)
      k_count_pairs<3><<<nbk, 256, 0, run>>>(P->desc.levels, ws.sstart, ws.tstart,
                                             &ws.geom->p2p_pairs);
    else
      k_count_pairs<2><<<nbk, 256, 0, run>>>(P->desc.levels, ws.sstart, ws.tstart,
                                             &ws.geom->p2p_pairs);
    ++nl;
  }
  if (split && (cudaEventRecord(P->ev_out, run) != cudaSuccess ||
                cudaStreamWaitEvent(st, P->ev_out, 0) != cudaSuccess))
    return FMM_ERR_CUDA;
  P->last_stream = st;
  P->last_geom = ws.geom;
  P->launches = first ? nl : P->launches + nl;
  return FMM_OK;
}

extern "C" int fmm_eval(fmm_plan_t P, int64_t n_src, const double* src, const double* w,
                        int64_t n_tgt, const double* tgt, double* phi, double* grad,
                        void* workspace, size_t wbytes, void* stream) {
  if (n_tgt > 0 && !phi) return FMM_ERR_ARG;
  return eval_internal(P, n_src, src, w, n_tgt, tgt, phi, grad, workspace, wbytes,
                       static_cast<cudaStream_t>(stream), true);
}

// ---- float32 entry: widen the inputs, evaluate, narrow the outputs ----------
__global__ void k_widen(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}
__global__ void k_narrow(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// float64 staging of an fmm_eval_f32 call (in front of the workspace proper)
struct F32Stage {
  size_t bytes;
  size_t src, w, tgt, phi, grad;  // byte offsets
};
static F32Stage f32_stage(const fmm_plan_s* P, int64_t n_src, int64_t n_tgt) {
  const int d = P->pd.d;
  const int cplx = P->pd.kernel == FMM_KERNEL_HELMHOLTZ ? 2 : 1;
  F32Stage f{};
  size_t o = 0;
  f.src = o;
  o += align_up(sizeof(double) * (size_t)std::max<int64_t>(n_src, 1) * d);
  f.w = o;
  o += align_up(sizeof(double) * (size_t)std::max<int64_t>(n_src, 1));
  f.tgt = o;
  o += align_up(sizeof(double) * (size_t)std::max<int64_t>(n_tgt, 1) * d);
  f.phi = o;
  o += align_up(sizeof(double) * (size_t)std::max<int64_t>(n_tgt, 1) * cplx);
  f.grad = o;
  o += align_up(sizeof(double) * (size_t)std::max<int64_t>(n_tgt, 1) * d * cplx);
  f.bytes = o;
  return f;
}

extern "C" int fmm_workspace_size_f32(fmm_plan_t P, int64_t n_src, int64_t n_tgt,
                                      size_t* bytes) {
  size_t b = 0;
  const int rc = fmm_workspace_size(P, n_src, n_tgt, &b);
  if (rc != FMM_OK) return rc;
  *bytes = b + f32_stage(P, n_src, n_tgt).bytes;
  return FMM_OK;
}

extern "C" int fmm_eval_f32(fmm_plan_t P, int64_t n_src, const float* src, const float* w,
                            int64_t n_tgt, const float* tgt, float* phi, float* grad,
                            void* workspace, size_t wbytes, void* stream) {
  if (!P || n_src < 0 || n_tgt < 0) return FMM_ERR_ARG;
  if (n_src > 0 && (!src || !w)) return FMM_ERR_ARG;
  if (n_tgt > 0 && (!tgt || !phi)) return FMM_ERR_ARG;
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign) return FMM_ERR_ARG;
  if (n_src > INT32_MAX / 2 || n_tgt > INT32_MAX / 2) return FMM_ERR_ARG;
  const F32Stage f = f32_stage(P, n_src, n_tgt);
  if (wbytes < f.bytes) return FMM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  double* s64 = reinterpret_cast<double*>(base + f.src);
  double* w64 = reinterpret_cast<double*>(base + f.w);
  double* t64 = reinterpret_cast<double*>(base + f.tgt);
  double* p64 = reinterpret_cast<double*>(base + f.phi);
  double* g64 = grad ? reinterpret_cast<double*>(base + f.grad) : nullptr;
  const int d = P->pd.d;
  const int cplx = P->pd.kernel == FMM_KERNEL_HELMHOLTZ ? 2 : 1;
  auto grid = [](int64_t n) { return (unsigned)((n + 255) / 256); };
  int nl = 0;
  if (n_src > 0) {
    k_widen<<<grid(n_src * d), 256, 0, st>>>(n_src * d, src, s64);
    k_widen<<<grid(n_src), 256, 0, st>>>(n_src, w, w64);
    nl += 2;
  }
  const bool same = tgt == src && n_tgt == n_src;  // one copy, one sort (as in fmm_eval)
  if (n_tgt > 0 && !same) {
    k_widen<<<grid(n_tgt * d), 256, 0, st>>>(n_tgt * d, tgt, t64);
    ++nl;
  }
  if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
  const int rc = eval_internal(P, n_src, s64, w64, n_tgt, same ? s64 : t64, p64, g64,
                               base + f.bytes, wbytes - f.bytes, st, true);
  if (rc != FMM_OK) return rc;
  if (n_tgt > 0) {
    k_narrow<<<grid(n_tgt * cplx), 256, 0, st>>>(n_tgt * cplx, p64, phi);
    ++nl;
    if (grad) {
      k_narrow<<<grid(n_tgt * d * cplx), 256, 0, st>>>(n_tgt * d * cplx, g64, grad);
      ++nl;
    }
  }
  P->launches += nl;
  return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

__global__ void k_scale_rows(int64_t n, int d, const double* s, double* g) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n * d) g[i] *= s[i / d];
}

__global__ void k_scale_rows_from(int64_t n, int d, const double* s, const double* g,
                                  double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n * d) out[i] = g[i] * s[i / d];
}

extern "C" int fmm_eval_backward(fmm_plan_t P, int64_t n_src, const double* src,
                                 const double* w, int64_t n_tgt, const double* tgt,
                                 const double* u, const double* grad_phi, double* grad_w,
                                 double* grad_src, double* grad_tgt, void* workspace,
                                 size_t wbytes, void* stream) {
  if (!P) return FMM_ERR_ARG;
  if (P->desc.levels < 0 || P->pd.kernel == FMM_KERNEL_HELMHOLTZ) return FMM_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int d = P->pd.d;
  int rc = FMM_OK;
  bool first = true;
  // transposed FMM: sources = targets with weights u, evaluated at the sources
  if (grad_w || grad_src) {
    if (n_src > 0 && !grad_w && !grad_src) return FMM_ERR_ARG;
    double* phi_out = grad_w;
    rc = eval_internal(P, n_tgt, tgt, u, n_src, src, phi_out, grad_src, workspace, wbytes, st,
                       first);
    if (rc != FMM_OK) return rc;
    first = false;
    if (grad_src && n_src > 0) {
      int64_t tot = n_src * d;
      k_scale_rows<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n_src, d, w, grad_src);
      P->launches++;
      if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    }
  }
  if (grad_tgt && grad_phi) {  // the forward's gradient: u * grad phi, no second FMM
    if (n_tgt > 0) {
      const int64_t tot = n_tgt * d;
      k_scale_rows_from<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n_tgt, d, u, grad_phi,
                                                                        grad_tgt);
      P->launches = first ? 1 : P->launches + 1;
      if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    }
  } else if (grad_tgt) {
    rc = eval_internal(P, n_src, src, w, n_tgt, tgt, nullptr, grad_tgt, workspace, wbytes, st,
                       first);
    if (rc != FMM_OK) return rc;
    if (n_tgt > 0) {
      int64_t tot = n_tgt * d;
      k_scale_rows<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n_tgt, d, u, grad_tgt);
      P->launches++;
      if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    }
  }
  return FMM_OK;
}

extern "C" int fmm_last_status(fmm_plan_t P) {
  if (!P) return FMM_ERR_ARG;
  if (!P->last_geom) return FMM_OK;
  if (cudaStreamSynchronize(P->last_stream) != cudaSuccess) return FMM_ERR_CUDA;
  Geom g;
  if (cudaMemcpy(&g, P->last_geom, sizeof(Geom), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FMM_ERR_CUDA;
  if (g.flag & 2) return FMM_ERR_TIMEOUT;
  if (g.flag & ~3) return FMM_ERR_INCOMPLETE;  // bit 4 (traversal stack) or any unknown bit
  if (g.flag & 1) return FMM_ERR_DOMAIN;
  return FMM_OK;
}

extern "C" const char* fmm_status_string(int s) {
  switch (s) {
    case FMM_OK: return "ok";
    case FMM_ERR_ARG: return "invalid argument";
    case FMM_ERR_UNSUPPORTED: return "unsupported kernel, dimension or PDE";
    case FMM_ERR_CUDA: return "CUDA runtime error";
    case FMM_ERR_NOMEM: return "out of memory";
    case FMM_ERR_TIMEOUT: return "bounded device wait gave up";
    case FMM_ERR_DOMAIN: return "point outside the root box (clamped)";
    case FMM_ERR_WORKSPACE: return "workspace too small";
    case FMM_ERR_INCOMPLETE: return "a fixed-size device structure overflowed (result incomplete)";
    default: return "unknown status";
  }
}
