// Host-side planner: pure integer structure work. Validates block structures,
// matches blocks by charge, groups them into charge sectors, builds the output
// structure in canonical order and the job tables that the device kernels run.
//
// Sec. II.A (block conservation rule sum_i s_i rho_i = n, lazy storage in one
// 1-D array) and Sec. II.B (fusion: nu = s_r (s_i rho + s_j rho'), D_nu =
// sum D_rho D_rho'; contraction = fuse -> multiply per sector -> unfuse, with
// the non-zero blocks precomputed) define what is planned here.
#include <algorithm>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <sstream>

#include "ytn_internal.hpp"

namespace ytn {

using Key = std::vector<int32_t>;

static inline int32_t reduce(int64_t v, int m) {
  if (m == 0) return (int32_t)v;
  int64_t r = v % m;
  return (int32_t)(r < 0 ? r + m : r);
}

static std::string keystr(const Key &k) {
  std::ostringstream os;
  os << "(";
  for (size_t i = 0; i < k.size(); i++) os << (i ? "," : "") << k[i];
  os << ")";
  return os.str();
}

// ---------------------------------------------------------------------------
// Loading and validating a ytn_struct
// ---------------------------------------------------------------------------

ytn_status load_struct(const ytn_struct *s, Tensor &T, std::string &err) {
  if (!s) { err = "null structure"; return YTN_E_INVALID; }
  if (s->sym.nsym < 1 || s->sym.nsym > YTN_MAX_SYM) { err = "nsym out of range"; return YTN_E_INVALID; }
  if (s->rank < 0 || s->rank > YTN_MAX_RANK) { err = "rank out of range"; return YTN_E_INVALID; }
  if (s->nblocks < 0 || s->size < 0) { err = "negative sizes"; return YTN_E_INVALID; }
  if (s->nblocks > 0 && s->rank > 0 && (!s->t || !s->D)) { err = "null block arrays"; return YTN_E_INVALID; }
  T = Tensor();
  if (s->dtype != YTN_REAL64 && s->dtype != YTN_COMPLEX128) { err = "unknown element type"; return YTN_E_INVALID; }
  T.dtype = s->dtype;
  T.nsym = s->sym.nsym;
  T.rank = s->rank;
  for (int c = 0; c < T.nsym; c++) {
    if (s->sym.mod[c] < 0 || s->sym.mod[c] == 1) { err = "modulus must be 0 (U(1)) or >= 2"; return YTN_E_INVALID; }
    T.mod[c] = s->sym.mod[c];
  }
  for (int c = 0; c < T.nsym; c++) T.n[c] = reduce(s->n[c], T.mod[c]);
  for (int i = 0; i < T.rank; i++) {
    if (s->sig[i] != 1 && s->sig[i] != -1) { err = "signature must be +1 or -1"; return YTN_E_INVALID; }
    T.sig[i] = s->sig[i];
  }
  T.nblocks = s->nblocks;
  const size_t nt = (size_t)T.nblocks * T.rank * T.nsym;
  const size_t nd = (size_t)T.nblocks * T.rank;
  T.t.assign(s->t ? s->t : nullptr, s->t ? s->t + nt : nullptr);
  T.D.assign(s->D ? s->D : nullptr, s->D ? s->D + nd : nullptr);
  T.size = s->size;
  T.off.resize(T.nblocks);
  int64_t acc = 0;
  for (int64_t b = 0; b < T.nblocks; b++) {
    int64_t e = 1;
    for (int i = 0; i < T.rank; i++) {
      int64_t d = T.dim(b, i);
      if (d < 1 || d > (int64_t)1 << 30) { err = "block dimension out of range"; return YTN_E_INVALID; }
      e *= d;
      if (e > ((int64_t)1 << 40)) { err = "block too large"; return YTN_E_INVALID; }
    }
    T.off[b] = s->off ? s->off[b] : acc;
    if (T.off[b] < 0 || T.off[b] + e > T.size) { err = "block outside the data buffer"; return YTN_E_INVALID; }
    acc += e;
  }
  // Z_m charges reduced; conservation; canonical order; one dimension per charge and leg.
  std::vector<std::map<Key, int64_t>> legdim(T.rank);
  for (int64_t b = 0; b < T.nblocks; b++) {
    int64_t tot[YTN_MAX_SYM] = {0};
    for (int i = 0; i < T.rank; i++) {
      const int32_t *q = T.charge(b, i);
      for (int c = 0; c < T.nsym; c++) {
        if (T.mod[c] && (q[c] < 0 || q[c] >= T.mod[c])) { err = "Z_m charge not reduced"; return YTN_E_INVALID; }
        tot[c] += (int64_t)T.sig[i] * q[c];
      }
      Key k(q, q + T.nsym);
      auto it = legdim[i].find(k);
      if (it == legdim[i].end()) legdim[i][k] = T.dim(b, i);
      else if (it->second != T.dim(b, i)) {
        err = "leg " + std::to_string(i) + " charge " + keystr(k) + " has two dimensions";
        return YTN_E_DIM_MISMATCH;
      }
    }
    for (int c = 0; c < T.nsym; c++)
      if (reduce(tot[c], T.mod[c]) != T.n[c]) {
        err = "block " + std::to_string(b) + " violates charge conservation";
        return YTN_E_CHARGE;
      }
    if (b > 0) {
      const int32_t *p = &T.t[(size_t)(b - 1) * T.rank * T.nsym];
      const int32_t *q = &T.t[(size_t)b * T.rank * T.nsym];
      if (!std::lexicographical_compare(p, p + T.rank * T.nsym, q, q + T.rank * T.nsym)) {
        err = "blocks not in strictly ascending canonical order";
        return YTN_E_INVALID;
      }
    }
  }
  if (T.rank == 0 && T.nblocks > 1) { err = "rank-0 tensor with more than one block"; return YTN_E_INVALID; }
  for (int i = 0; i < T.rank; i++) {
    const ytn_fusion *f = s->fus[i];
    if (!f) continue;
    // a record with no rows (the fusion of a tensor without blocks) may have null arrays
    if (f->nlegs < 2 || f->nlegs > YTN_MAX_RANK || f->nentries < 0 ||
        (f->nentries > 0 && (!f->nu || !f->t || !f->D))) {
      err = "malformed fusion record";
      return YTN_E_INVALID;
    }
    auto F = std::make_shared<Fusion>();
    F->nlegs = f->nlegs;
    for (int j = 0; j < f->nlegs; j++) {
      if (f->sig[j] != 1 && f->sig[j] != -1) { err = "fusion record signature"; return YTN_E_INVALID; }
      F->sig[j] = f->sig[j];
    }
    F->nentries = f->nentries;
    if (f->nentries > 0) {
      F->nu.assign(f->nu, f->nu + f->nentries * T.nsym);
      F->t.assign(f->t, f->t + f->nentries * f->nlegs * T.nsym);
      F->D.assign(f->D, f->D + f->nentries * f->nlegs);
    }
    // entries sorted by (nu, constituent charges); each row consistent with F2
    std::map<Key, int64_t> dnu;
    for (int64_t e = 0; e < F->nentries; e++) {
      int64_t tot[YTN_MAX_SYM] = {0};
      for (int j = 0; j < F->nlegs; j++)
        for (int c = 0; c < T.nsym; c++) tot[c] += (int64_t)F->sig[j] * F->t[(e * F->nlegs + j) * T.nsym + c];
      int64_t sz = 1;
      for (int j = 0; j < F->nlegs; j++) {
        if (F->D[e * F->nlegs + j] < 1) { err = "fusion record dimension"; return YTN_E_INVALID; }
        sz *= F->D[e * F->nlegs + j];
      }
      for (int c = 0; c < T.nsym; c++)
        if (reduce((int64_t)T.sig[i] * tot[c], T.mod[c]) != F->nu[e * T.nsym + c]) {
          err = "fusion record charge does not follow nu = s_r sum_i s_i rho_i";
          return YTN_E_INVALID;
        }
      Key k(&F->nu[e * T.nsym], &F->nu[e * T.nsym] + T.nsym);
      dnu[k] += sz;
      if (e > 0) {
        Key a(&F->nu[(e - 1) * T.nsym], &F->nu[(e - 1) * T.nsym] + T.nsym);
        a.insert(a.end(), &F->t[(e - 1) * F->nlegs * T.nsym], &F->t[e * F->nlegs * T.nsym]);
        Key bk = k;
        bk.insert(bk.end(), &F->t[e * F->nlegs * T.nsym], &F->t[(e + 1) * F->nlegs * T.nsym]);
        if (!(a < bk)) { err = "fusion record rows not in ascending order"; return YTN_E_INVALID; }
      }
    }
    for (auto &kv : legdim[i]) {
      auto it = dnu.find(kv.first);
      if (it == dnu.end() || it->second != kv.second) {
        err = "fused leg " + std::to_string(i) + " block dimension does not match its record";
        return YTN_E_INVALID;
      }
    }
    T.fus[i] = F;
  }
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------

static Key sub_charges(const Tensor &T, int64_t b, const std::vector<int> &legs) {
  Key k;
  k.reserve(legs.size() * T.nsym);
  for (int l : legs) {
    const int32_t *q = T.charge(b, l);
    k.insert(k.end(), q, q + T.nsym);
  }
  return k;
}

static int64_t sub_elems(const Tensor &T, int64_t b, const std::vector<int> &legs) {
  int64_t e = 1;
  for (int l : legs) e *= T.dim(b, l);
  return e;
}

static std::map<Key, int64_t> leg_dims(const Tensor &T, int leg) {
  std::map<Key, int64_t> m;
  for (int64_t b = 0; b < T.nblocks; b++) {
    const int32_t *q = T.charge(b, leg);
    m[Key(q, q + T.nsym)] = T.dim(b, leg);
  }
  if (T.fus[leg]) {
    const Fusion &F = *T.fus[leg];
    std::map<Key, int64_t> dnu;
    for (int64_t e = 0; e < F.nentries; e++) {
      int64_t sz = 1;
      for (int j = 0; j < F.nlegs; j++) sz *= F.D[e * F.nlegs + j];
      dnu[Key(&F.nu[e * T.nsym], &F.nu[e * T.nsym] + T.nsym)] += sz;
    }
    for (auto &kv : dnu) m.emplace(kv.first, kv.second);
  }
  return m;
}

static bool fusion_conj_equal(const Fusion &a, const Fusion &b) {
  if (a.nlegs != b.nlegs || a.nentries != b.nentries) return false;
  for (int j = 0; j < a.nlegs; j++)
    if (a.sig[j] != -b.sig[j]) return false;
  return a.nu == b.nu && a.t == b.t && a.D == b.D;
}

// Paired legs (contraction or trace) must be compatible: opposite signatures,
// one dimension per charge present on both, conjugate fusion records.
static ytn_status check_pair(const Tensor &A, int a, const Tensor &B, int b, std::string &err) {
  if (A.sig[a] != -B.sig[b]) {
    err = "paired legs " + std::to_string(a) + "/" + std::to_string(b) + " have equal signatures";
    return YTN_E_SIGNATURE;
  }
  auto da = leg_dims(A, a), db = leg_dims(B, b);
  for (auto &kv : da) {
    auto it = db.find(kv.first);
    if (it != db.end() && it->second != kv.second) {
      err = "charge " + keystr(kv.first) + " has dimension " + std::to_string(kv.second) + " vs " +
            std::to_string(it->second) + " on paired legs";
      return YTN_E_DIM_MISMATCH;
    }
  }
  const bool fa = (bool)A.fus[a], fb = (bool)B.fus[b];
  if (fa != fb) { err = "a fused leg is paired with a plain leg"; return YTN_E_FUSION_MISMATCH; }
  if (fa && !fusion_conj_equal(*A.fus[a], *B.fus[b])) {
    err = "fusion records of paired legs differ";
    return YTN_E_FUSION_MISMATCH;
  }
  return YTN_OK;
}

// Row-major element strides of block b.
static std::vector<int64_t> block_strides(const Tensor &T, int64_t b) {
  if (!T.bstr.empty()) return std::vector<int64_t>(T.bstr.begin() + b * T.rank, T.bstr.begin() + (b + 1) * T.rank);
  std::vector<int64_t> st(T.rank);
  int64_t acc = 1;
  for (int i = T.rank - 1; i >= 0; i--) {
    st[i] = acc;
    acc *= T.dim(b, i);
  }
  return st;
}

struct Dim {
  int64_t ext, sst, dst;
};

// Division by d >= 1 of any n < 2^31 as (n + umulhi(n, m)) >> sh: with
// l = ceil(log2 d), M = ceil(2^(32 + l) / d) in [2^32, 2^33), m = M - 2^32 and
// sh = l, the sum is floor(n M / 2^32) and the quotient is exact, because
// M d - 2^(32 + l) < d makes the excess of n M / 2^(32 + l) over n / d smaller
// than n / 2^(32 + l) < 2^-(l + 1) < 1 / d. d = 1 gives m = 0, sh = 0.
static void division_magic(int64_t d, uint32_t &m, uint8_t &sh) {
  int l = 0;
  while ((int64_t(1) << l) < d) l++;
  const uint64_t num = uint64_t(1) << (32 + l);   // l <= 31: no overflow below
  const uint64_t M = (num + (uint64_t)d - 1) / (uint64_t)d;
  m = (uint32_t)(M - (uint64_t(1) << 32));
  sh = (uint8_t)l;
}

// Drop unit dims and merge neighbours that are contiguous in both layouts
// (dims listed outer -> inner in the order that is kept).
static std::vector<Dim> merge_dims(const std::vector<Dim> &dims) {
  std::vector<Dim> m;
  for (auto &d : dims) {
    if (d.ext == 1) continue;
    if (!m.empty() && m.back().sst == d.sst * d.ext && m.back().dst == d.dst * d.ext) {
      m.back().ext *= d.ext;
      m.back().sst = d.sst;
      m.back().dst = d.dst;
    } else {
      m.push_back(d);
    }
  }
  return m;
}

// True if the dims fill a dense row-major range on the source (or destination)
// side, starting at its origin.
static bool side_dense(const std::vector<Dim> &dims, bool src) {
  std::vector<std::pair<int64_t, int64_t>> v;   // (stride, extent)
  for (auto &d : dims) v.push_back({src ? d.sst : d.dst, d.ext});
  std::sort(v.begin(), v.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
  int64_t expect = 1;
  for (size_t i = v.size(); i-- > 0;) {
    if (v[i].first != expect) return false;
    expect *= v[i].second;
  }
  return true;
}

// One staged job: `dims` (ext, local stride, global stride) of a piece whose
// dense side starts at d_off and strided side at g_off.
static ytn_status push_piece(ytn_plan_t *p, std::vector<Dim> dims, int mode, int64_t g_off, int64_t d_off,
                             std::string &err, int negate = 0) {
  // enumeration order: strided (global) side outer -> inner
  std::stable_sort(dims.begin(), dims.end(), [](const Dim &a, const Dim &b) { return a.dst > b.dst; });
  std::vector<Dim> m = merge_dims(dims);
  if (m.empty()) m.push_back({1, 1, 1});
  if ((int)m.size() > kMaxCopyDims) {
    err = "copy job needs more than 8 dimensions";
    return YTN_E_UNSUPPORTED;
  }
  if (negate == 2 && mode != 2) {   // the parity rule needs the source side dense
    err = "imaginary-part negation of a copy without a dense source";
    return YTN_E_UNSUPPORTED;
  }
  CopyJob J;
  std::memset(&J, 0, sizeof(J));
  J.g_off = g_off;
  J.d_off = d_off;
  J.nd = (int32_t)m.size();
  J.mode = mode;
  J.negate = negate;
  int64_t size = 1;
  // dims right-aligned in the kMaxCopyDims slots; the outer slots are unit dims
  const int o = kMaxCopyDims - J.nd;
  for (int i = 0; i < kMaxCopyDims; i++) {
    J.ext[i] = 1;
    division_magic(1, J.mag[i], J.shf[i]);
  }
  for (int i = 0; i < J.nd; i++) {
    if (m[i].dst > INT32_MAX) {
      err = "copy job stride exceeds 32 bits";
      return YTN_E_UNSUPPORTED;
    }
    J.ext[o + i] = (int32_t)m[i].ext;
    J.lstr[o + i] = (int32_t)m[i].sst;
    J.gstr[o + i] = (int32_t)m[i].dst;
    division_magic(m[i].ext, J.mag[o + i], J.shf[o + i]);
    size *= m[i].ext;
  }
  J.size = (int32_t)size;
  p->jobs.push_back(J);
  return YTN_OK;
}

// A block copy (dims outer -> inner in destination order, strides of both
// sides) becomes staged jobs of at most kStageElems elements. One side is a
// dense range (the whole block on the tensor side); it is cut into contiguous
// pieces by fixing its outer indices and splitting the next one.
static ytn_status add_copy_raw(ytn_plan_t *p, const std::vector<Dim> &dims, int64_t src_off, int64_t dst_off,
                               std::string &err, int negate);

// A block copy in elements; for complex tensors moved whole (p->cw == 2) every
// element is a pair of doubles: strides and offsets double and an innermost
// component dim (2, 1, 1) is added.
static ytn_status add_copy(ytn_plan_t *p, const std::vector<Dim> &dims, int64_t src_off, int64_t dst_off,
                           std::string &err, int negate = 0) {
  if (p->cw != 2) return add_copy_raw(p, dims, src_off, dst_off, err, negate);
  std::vector<Dim> d2;
  for (const Dim &d : dims) d2.push_back({d.ext, 2 * d.sst, 2 * d.dst});
  d2.push_back({2, 1, 1});
  return add_copy_raw(p, d2, 2 * src_off, 2 * dst_off, err, negate);
}

static ytn_status add_copy_raw(ytn_plan_t *p, const std::vector<Dim> &dims, int64_t src_off, int64_t dst_off,
                               std::string &err, int negate) {
  std::vector<Dim> v;
  for (auto &d : dims)
    if (d.ext != 1) v.push_back(d);
  int mode;
  int64_t g0, d0;
  // local form: ext, dense-side stride (sst field), strided-side stride (dst field)
  std::vector<Dim> loc;
  if (side_dense(v, true)) {
    mode = 2;   // dense source: read linearly, written in destination order
    for (auto &d : v) loc.push_back({d.ext, d.sst, d.dst});
    d0 = src_off;
    g0 = dst_off;
  } else if (side_dense(v, false)) {
    mode = 3;   // dense destination: read in source order, written linearly
    for (auto &d : v) loc.push_back({d.ext, d.dst, d.sst});
    d0 = dst_off;
    g0 = src_off;
  } else {
    // neither side is one contiguous range (a strided view of a block): on the
    // side with the longer contiguous innermost run, fix the outer indices and
    // copy each run (a single element when neither side has one)
    auto suffix = [&](bool src, std::vector<Dim> &srt, int64_t &run) {
      srt = v;
      std::sort(srt.begin(), srt.end(),
                [src](const Dim &a, const Dim &b) { return src ? a.sst > b.sst : a.dst > b.dst; });
      size_t k = srt.size();
      run = 1;
      while (k > 0 && (src ? srt[k - 1].sst : srt[k - 1].dst) == run) {
        run *= srt[k - 1].ext;
        k--;
      }
      return k;
    };
    std::vector<Dim> ss, sd;
    int64_t rs, rd;
    const size_t ks_ = suffix(true, ss, rs), kd_ = suffix(false, sd, rd);
    const bool use_src = rs >= rd;
    const std::vector<Dim> &srt = use_src ? ss : sd;
    const size_t k = use_src ? ks_ : kd_;
    std::vector<Dim> inner(srt.begin() + k, srt.end());
    std::vector<int64_t> idx(k, 0);
    for (;;) {
      int64_t so = src_off, dof = dst_off;
      for (size_t i = 0; i < k; i++) {
        so += idx[i] * srt[i].sst;
        dof += idx[i] * srt[i].dst;
      }
      ytn_status s = add_copy_raw(p, inner, so, dof, err, negate);
      if (s != YTN_OK) return s;
      size_t i = k;
      while (i > 0 && ++idx[i - 1] == srt[i - 1].ext) idx[--i] = 0;
      if (i == 0) break;
    }
    return YTN_OK;
  }
  // dense-side order, outer -> inner
  std::sort(loc.begin(), loc.end(), [](const Dim &a, const Dim &b) { return a.sst > b.sst; });
  const int n = (int)loc.size();
  // k: outermost dim whose inner product fits a piece
  int64_t inner = 1;
  int k = n;
  while (k > 0 && inner * loc[k - 1].ext <= kStageElems) {
    inner *= loc[k - 1].ext;
    k--;
  }
  if (k == 0) return push_piece(p, loc, mode, g0, d0, err, negate);
  // dims [0, k-1) are fixed per piece, dim k-1 is split into runs of `c`
  const int ks = k - 1;
  const int64_t c = std::max<int64_t>(1, kStageElems / inner);
  std::vector<int64_t> idx(ks, 0);
  for (;;) {
    int64_t go = g0, dof = d0;
    for (int i = 0; i < ks; i++) {
      go += idx[i] * loc[i].dst;
      dof += idx[i] * loc[i].sst;
    }
    for (int64_t a = 0; a < loc[ks].ext; a += c) {
      std::vector<Dim> piece(loc.begin() + ks, loc.end());
      piece[0].ext = std::min(c, loc[ks].ext - a);
      ytn_status s = push_piece(p, piece, mode, go + a * loc[ks].dst, dof + a * loc[ks].sst, err, negate);
      if (s != YTN_OK) return s;
    }
    int i = ks - 1;
    for (; i >= 0; i--) {
      if (++idx[i] < loc[i].ext) break;
      idx[i] = 0;
    }
    if (i < 0) break;
  }
  return YTN_OK;
}

// Pack jobs [j0, j1) into CTA work items: runs of consecutive jobs of one
// mode, at most kStageElems elements and kStageJobs jobs each; the item's
// dimension count is the largest of its jobs' (the others have unit dims in
// the outer slots).
static void make_items(ytn_plan_t *p, size_t j0, size_t j1) {
  size_t j = j0;
  while (j < j1) {
    const CopyJob &F = p->jobs[j];
    size_t k = j;
    int32_t tot = 0, nd = 1;
    while (k < j1 && k - j < (size_t)kStageJobs && p->jobs[k].mode == F.mode &&
           tot + p->jobs[k].size <= kStageElems) {
      p->jobs[k].p = tot;
      tot += p->jobs[k].size;
      nd = std::max(nd, p->jobs[k].nd);
      k++;
    }
    CopyItem it;
    it.job = (int32_t)j;
    it.njobs = (int32_t)(k - j);
    it.total = tot;
    it.kind = nd | (F.mode << 8);
    p->items.push_back(it);
    j = k;
  }
}

static void copy_fusion(const Fusion *f, std::shared_ptr<Fusion> &dst) {
  dst = f ? std::make_shared<Fusion>(*f) : nullptr;
}

// Sort output blocks canonically and assign packed offsets.
struct OutBlock {
  Key key;                  // flattened charges, rank * nsym
  std::vector<int64_t> D;   // rank
  int64_t id;               // caller's handle
};

static void finalize_out(Tensor &C, std::vector<OutBlock> &blocks, std::vector<int64_t> &offset_of_id) {
  std::sort(blocks.begin(), blocks.end(), [](const OutBlock &a, const OutBlock &b) { return a.key < b.key; });
  C.nblocks = (int64_t)blocks.size();
  C.t.clear();
  C.D.clear();
  C.off.clear();
  int64_t acc = 0;
  offset_of_id.assign(blocks.size(), 0);
  for (auto &ob : blocks) {
    C.t.insert(C.t.end(), ob.key.begin(), ob.key.end());
    C.D.insert(C.D.end(), ob.D.begin(), ob.D.end());
    C.off.push_back(acc);
    offset_of_id[ob.id] = acc;
    int64_t e = 1;
    for (auto d : ob.D) e *= d;
    acc += e;
  }
  C.size = acc;
}

// ---------------------------------------------------------------------------
// Tensordot
// ---------------------------------------------------------------------------

// A view of T with the fused legs `legs` replaced by their constituents (the
// unfusion of Sec. II.B without moving data): every recorded sub-block of every
// stored fused block becomes a block of the view, addressed inside the fused
// block through explicit strides. Blocks are put in canonical order.
static ytn_status unfuse_view(const Tensor &T, const std::vector<int> &legs, Tensor &V, std::string &err) {
  std::vector<char> isun(T.rank, 0);
  int rank = T.rank;
  for (int l : legs) {
    isun[l] = 1;
    rank += T.fus[l]->nlegs - 1;
  }
  if (rank > YTN_MAX_RANK) { err = "unfused view exceeds the maximum rank"; return YTN_E_UNSUPPORTED; }
  const int nsym = T.nsym;
  V = Tensor();
  V.dtype = T.dtype;
  V.nsym = nsym;
  std::memcpy(V.mod, T.mod, sizeof(V.mod));
  std::memcpy(V.n, T.n, sizeof(V.n));
  V.rank = rank;
  V.size = T.size;
  for (int l = 0, r = 0; l < T.rank; l++) {
    if (isun[l]) {
      for (int j = 0; j < T.fus[l]->nlegs; j++) V.sig[r++] = T.fus[l]->sig[j];
    } else {
      V.fus[r] = T.fus[l];
      V.sig[r++] = T.sig[l];
    }
  }
  // per fused leg and fused charge: the record's rows with their offsets
  struct Row { int64_t e, off; };
  std::vector<std::map<Key, std::vector<Row>>> rows(T.rank);
  for (int l : legs) {
    const Fusion &F = *T.fus[l];
    for (int64_t e = 0; e < F.nentries; e++) {
      Key nu(&F.nu[e * nsym], &F.nu[e * nsym] + nsym);
      auto &lst = rows[l][nu];
      int64_t off = 0;
      if (!lst.empty()) {
        const Row &pr = lst.back();
        int64_t sz = 1;
        for (int j = 0; j < F.nlegs; j++) sz *= F.D[pr.e * F.nlegs + j];
        off = pr.off + sz;
      }
      lst.push_back({e, off});
    }
  }
  struct Sub { Key key; std::vector<int64_t> D, st; int64_t off; };
  std::vector<Sub> subs;
  for (int64_t b = 0; b < T.nblocks; b++) {
    const auto st = block_strides(T, b);
    std::vector<const std::vector<Row> *> ch(T.rank, nullptr);
    bool ok = true;
    for (int l : legs) {
      const int32_t *q = T.charge(b, l);
      auto it = rows[l].find(Key(q, q + nsym));
      if (it == rows[l].end()) { ok = false; break; }   // not in the record: checked at load
      ch[l] = &it->second;
    }
    if (!ok) { err = "fused block without a record row"; return YTN_E_INVALID; }
    std::vector<size_t> pick(T.rank, 0);
    for (;;) {
      Sub sb;
      sb.off = T.off[b];
      for (int l = 0; l < T.rank; l++) {
        if (!isun[l]) {
          const int32_t *q = T.charge(b, l);
          sb.key.insert(sb.key.end(), q, q + nsym);
          sb.D.push_back(T.dim(b, l));
          sb.st.push_back(st[l]);
          continue;
        }
        const Fusion &F = *T.fus[l];
        const Row &rw = (*ch[l])[pick[l]];
        sb.off += rw.off * st[l];
        int64_t inner = st[l];
        std::vector<int64_t> cst(F.nlegs);
        for (int j = F.nlegs - 1; j >= 0; j--) {
          cst[j] = inner;
          inner *= F.D[rw.e * F.nlegs + j];
        }
        for (int j = 0; j < F.nlegs; j++) {
          const int32_t *q = &F.t[(rw.e * F.nlegs + j) * nsym];
          sb.key.insert(sb.key.end(), q, q + nsym);
          sb.D.push_back(F.D[rw.e * F.nlegs + j]);
          sb.st.push_back(cst[j]);
        }
      }
      subs.push_back(std::move(sb));
      int l = T.rank - 1;
      for (; l >= 0; l--) {
        if (!isun[l]) continue;
        if (++pick[l] < ch[l]->size()) break;
        pick[l] = 0;
      }
      if (l < 0) break;
    }
  }
  std::sort(subs.begin(), subs.end(), [](const Sub &x, const Sub &y) { return x.key < y.key; });
  V.nblocks = (int64_t)subs.size();
  for (auto &sb : subs) {
    V.t.insert(V.t.end(), sb.key.begin(), sb.key.end());
    V.D.insert(V.D.end(), sb.D.begin(), sb.D.end());
    V.bstr.insert(V.bstr.end(), sb.st.begin(), sb.st.end());
    V.off.push_back(sb.off);
  }
  return YTN_OK;
}

// Contracted fused legs with different fusion histories (Sec. II.B footnote):
// resolvable when both come from the same number of constituent legs with
// opposite signatures and agree on the dimensions of every constituent charge
// tuple both records list. A tuple missing on one side is a zero sub-block, so
// the contraction runs over the constituents of unfused views of both tensors.
static ytn_status check_resolvable(const Fusion &a, const Fusion &b, int nsym, std::string &err) {
  if (a.nlegs != b.nlegs) { err = "contracted fused legs come from different constituent legs"; return YTN_E_FUSION_MISMATCH; }
  for (int j = 0; j < a.nlegs; j++)
    if (a.sig[j] != -b.sig[j]) { err = "contracted fused legs come from different constituent legs"; return YTN_E_FUSION_MISMATCH; }
  std::map<Key, std::vector<int64_t>> da;
  const int64_t w = (int64_t)a.nlegs * nsym;
  for (int64_t e = 0; e < a.nentries; e++)
    da[Key(&a.t[e * w], &a.t[e * w] + w)] = std::vector<int64_t>(&a.D[e * a.nlegs], &a.D[e * a.nlegs] + a.nlegs);
  for (int64_t e = 0; e < b.nentries; e++) {
    auto it = da.find(Key(&b.t[e * w], &b.t[e * w] + w));
    if (it != da.end() && it->second != std::vector<int64_t>(&b.D[e * b.nlegs], &b.D[e * b.nlegs] + b.nlegs)) {
      err = "a constituent charge tuple has different dimensions on the contracted fused legs";
      return YTN_E_DIM_MISMATCH;
    }
  }
  return YTN_OK;
}

// One sector of a contraction while it is being planned: its contracted charge
// tuples x (with |x|), its rows I (with |I| and one A block carrying it) and its
// columns J (with |J| and one B block).
struct SB {
  std::map<Key, int64_t> xs;
  std::map<Key, std::pair<int64_t, int64_t>> rows;
  std::map<Key, std::pair<int64_t, int64_t>> cols;
};

// Partition of one contraction over p->shard_world ranks (its sectors are
// independent matrix products, and each block of C lies in exactly one sector):
// the work units are whole sectors, except that a sector above a quarter of a
// rank's share is cut into runs of consecutive rows I of about that size; the
// units go to ranks by longest-processing-time first (largest useful FLOPs first,
// each to the least loaded rank, ties to the lower rank; units of equal FLOPs in
// sector and row order), the same on every rank since it is integer structure
// and a fixed order. The plan keeps p->shard_rank's rows of each sector (A and B
// stay whole; C's blocks are those of the kept rows) and its useful FLOPs.
static void shard_sectors(ytn_plan_t *p, const Tensor &A, const Tensor &B,
                          std::map<Key, std::vector<int64_t>> &Ax, std::map<Key, std::vector<int64_t>> &Bx,
                          const std::vector<int> &freeA, const std::vector<int> &freeB, std::map<Key, SB> &secs) {
  const int world = p->shard_world, rank = p->shard_rank;
  // useful FLOPs per row of each sector: 2 |I| |x| sum_{B(x, J)} |J| over the x of A(I, x)
  std::vector<std::vector<double>> row_fl;
  double total = 0;
  for (auto &kv : secs) {
    const SB &sb = kv.second;
    std::map<Key, size_t> ridx;
    for (auto &r : sb.rows) ridx.emplace(r.first, ridx.size());
    std::vector<double> fl(sb.rows.size(), 0.0);
    for (auto &x : sb.xs) {
      double nj = 0;
      for (int64_t b : Bx[x.first]) nj += (double)sub_elems(B, b, freeB);
      for (int64_t a : Ax[x.first]) {
        auto it = ridx.find(sub_charges(A, a, freeA));
        if (it != ridx.end()) fl[it->second] += 2.0 * (double)sub_elems(A, a, freeA) * (double)x.second * nj;
      }
    }
    for (double f : fl) total += f;
    row_fl.push_back(std::move(fl));
  }
  struct Unit { size_t sec, r0, r1; double fl; };
  std::vector<Unit> units;
  const double cap = total / world / 4.0;
  for (size_t si = 0; si < row_fl.size(); si++) {
    const auto &fl = row_fl[si];
    double sf = 0;
    for (double f : fl) sf += f;
    if (sf <= cap || fl.size() < 2) {
      units.push_back({si, 0, fl.size(), sf});
      continue;
    }
    size_t r0 = 0;
    double acc = 0;
    for (size_t r = 0; r < fl.size(); r++) {
      acc += fl[r];
      if (acc >= cap || r + 1 == fl.size()) {
        units.push_back({si, r0, r + 1, acc});
        r0 = r + 1;
        acc = 0;
      }
    }
  }
  std::stable_sort(units.begin(), units.end(), [](const Unit &x, const Unit &y) { return x.fl > y.fl; });
  std::vector<double> load(world, 0.0);
  std::vector<std::vector<std::pair<size_t, size_t>>> mine(row_fl.size());
  for (const Unit &u : units) {
    int best = 0;
    for (int r = 1; r < world; r++)
      if (load[r] < load[best]) best = r;
    load[best] += u.fl;
    if (best == rank) mine[u.sec].push_back({u.r0, u.r1});
  }
  // keep this rank's rows; drop sectors with none
  double kept = 0;
  size_t si = 0;
  for (auto it = secs.begin(); it != secs.end(); si++) {
    auto &ranges = mine[si];
    if (ranges.empty()) {
      it = secs.erase(it);
      continue;
    }
    std::vector<char> keep(row_fl[si].size(), 0);
    for (auto &rg : ranges)
      for (size_t r = rg.first; r < rg.second; r++) keep[r] = 1;
    size_t r = 0;
    for (auto rit = it->second.rows.begin(); rit != it->second.rows.end(); r++) {
      if (keep[r]) {
        kept += row_fl[si][r];
        ++rit;
      } else {
        rit = it->second.rows.erase(rit);
      }
    }
    ++it;
  }
  p->flops = kept * p->ca * p->cb;
}

ytn_status plan_tensordot(ytn_plan_t *p, const Tensor &A, const Tensor &B, int naxes,
                          const int *axa_in, const int *axb_in, std::string &err) {
  if (A.nsym != B.nsym || std::memcmp(A.mod, B.mod, sizeof(A.mod)) != 0) {
    err = "tensors have different symmetries";
    return YTN_E_INVALID;
  }
  if (naxes < 0 || naxes > A.rank || naxes > B.rank) { err = "naxes out of range"; return YTN_E_INVALID; }
  std::vector<int> axa(axa_in, axa_in + naxes), axb(axb_in, axb_in + naxes);
  {
    std::set<int> sa(axa.begin(), axa.end()), sb(axb.begin(), axb.end());
    if ((int)sa.size() != naxes || (int)sb.size() != naxes) { err = "repeated axis"; return YTN_E_INVALID; }
    for (int k = 0; k < naxes; k++)
      if (axa[k] < 0 || axa[k] >= A.rank || axb[k] < 0 || axb[k] >= B.rank) {
        err = "axis out of range";
        return YTN_E_INVALID;
      }
  }
  if (A.rank + B.rank - 2 * naxes > YTN_MAX_RANK) { err = "output rank too large"; return YTN_E_UNSUPPORTED; }
  {
    std::vector<int> ua, ub;
    for (int k = 0; k < naxes; k++) {
      const int a = axa[k], b = axb[k];
      if (!A.fus[a] || !B.fus[b] || fusion_conj_equal(*A.fus[a], *B.fus[b])) continue;
      if (A.sig[a] != -B.sig[b]) {
        err = "paired legs " + std::to_string(a) + "/" + std::to_string(b) + " have equal signatures";
        return YTN_E_SIGNATURE;
      }
      ytn_status st = check_resolvable(*A.fus[a], *B.fus[b], A.nsym, err);
      if (st != YTN_OK) return st;
      ua.push_back(a);
      ub.push_back(b);
    }
    if (!ua.empty()) {
      Tensor VA, VB;
      ytn_status st = unfuse_view(A, ua, VA, err);
      if (st == YTN_OK) st = unfuse_view(B, ub, VB, err);
      if (st != YTN_OK) return st;
      auto expand = [](const Tensor &T, const std::vector<int> &un, const std::vector<int> &ax) {
        std::vector<std::vector<int>> pos(T.rank);
        for (int l = 0, r = 0; l < T.rank; l++) {
          const int n = std::find(un.begin(), un.end(), l) != un.end() ? T.fus[l]->nlegs : 1;
          for (int j = 0; j < n; j++) pos[l].push_back(r++);
        }
        std::vector<int> out;
        for (int a : ax) out.insert(out.end(), pos[a].begin(), pos[a].end());
        return out;
      };
      const std::vector<int> xa = expand(A, ua, axa), xb = expand(B, ub, axb);
      if ((int)xa.size() > YTN_MAX_RANK) { err = "unfused view exceeds the maximum rank"; return YTN_E_UNSUPPORTED; }
      return plan_tensordot(p, VA, VB, (int)xa.size(), xa.data(), xb.data(), err);
    }
  }
  for (int k = 0; k < naxes; k++) {
    ytn_status st = check_pair(A, axa[k], B, axb[k], err);
    if (st != YTN_OK) return st;
  }
  const int nsym = A.nsym;
  std::vector<int> freeA, freeB;
  for (int i = 0; i < A.rank; i++)
    if (std::find(axa.begin(), axa.end(), i) == axa.end()) freeA.push_back(i);
  for (int i = 0; i < B.rank; i++)
    if (std::find(axb.begin(), axb.end(), i) == axb.end()) freeB.push_back(i);

  // Complex operands: each becomes a real sector matrix twice as tall (A: rows of
  // the real parts, then of the imaginary parts) or twice as wide (B: columns of
  // real, then imaginary parts), so that one real grouped GEMM gives the four
  // products re.re, re.im, im.re, im.im as quadrants of C_q; the scatter combines
  // them into complex C (re = P00 - P11, im = P01 + P10).
  const int ca = A.dtype == YTN_COMPLEX128 ? 2 : 1, cb = B.dtype == YTN_COMPLEX128 ? 2 : 1;
  p->ca = ca;
  p->cb = cb;

  // Output tensor: A's free legs then B's; n_C = n_A + n_B.
  Tensor &C = p->out;
  C = Tensor();
  C.dtype = ca * cb > 1 ? YTN_COMPLEX128 : YTN_REAL64;
  C.nsym = nsym;
  std::memcpy(C.mod, A.mod, sizeof(C.mod));
  C.rank = (int)(freeA.size() + freeB.size());
  for (size_t i = 0; i < freeA.size(); i++) {
    C.sig[i] = A.sig[freeA[i]];
    copy_fusion(A.fus[freeA[i]].get(), C.fus[i]);
  }
  for (size_t i = 0; i < freeB.size(); i++) {
    C.sig[freeA.size() + i] = B.sig[freeB[i]];
    copy_fusion(B.fus[freeB[i]].get(), C.fus[freeA.size() + i]);
  }
  for (int c = 0; c < nsym; c++) C.n[c] = reduce((int64_t)A.n[c] + B.n[c], A.mod[c]);

  // Match blocks on the contracted charges x (in the order of axa / axb).
  std::map<Key, std::vector<int64_t>> Ax, Bx;
  for (int64_t b = 0; b < A.nblocks; b++) Ax[sub_charges(A, b, axa)].push_back(b);
  for (int64_t b = 0; b < B.nblocks; b++) Bx[sub_charges(B, b, axb)].push_back(b);

  // Sector key q = sum_k s_A[axa_k] x_k (reduced): every x, every row I of A and
  // every column J of B belongs to exactly one sector.
  std::map<Key, SB> secs;
  double flops = 0;
  for (auto &kv : Ax) {
    auto itb = Bx.find(kv.first);
    if (itb == Bx.end()) continue;
    Key q(nsym, 0);
    for (int k = 0; k < naxes; k++)
      for (int c = 0; c < nsym; c++)
        q[c] = reduce((int64_t)q[c] + (int64_t)A.sig[axa[k]] * kv.first[k * nsym + c], A.mod[c]);
    SB &s = secs[q];
    const int64_t b0 = kv.second[0];
    const int64_t kx = sub_elems(A, b0, axa);
    s.xs[kv.first] = kx;
    double si = 0, sj = 0;
    for (int64_t a : kv.second) {
      const int64_t ni = sub_elems(A, a, freeA);
      s.rows.emplace(sub_charges(A, a, freeA), std::make_pair(ni, a));
      si += (double)ni;
    }
    for (int64_t b : itb->second) {
      const int64_t nj = sub_elems(B, b, freeB);
      s.cols.emplace(sub_charges(B, b, freeB), std::make_pair(nj, b));
      sj += (double)nj;
    }
    flops += 2.0 * si * (double)kx * sj;
  }
  p->flops = flops * ca * cb;
  if (p->shard_world > 1) shard_sectors(p, A, B, Ax, Bx, freeA, freeB, secs);

  // Sector geometry: rows, K and columns in ascending charge order.
  struct SG {
    std::map<Key, int64_t> row_off, col_off, x_off;
    int64_t M = 0, N = 0, K = 0;
  };
  std::vector<SG> geo;
  std::vector<const SB *> sbs;
  for (auto &kv : secs) {
    SG g;
    for (auto &r : kv.second.rows) { g.row_off[r.first] = g.M; g.M += r.second.first; }
    for (auto &c : kv.second.cols) { g.col_off[c.first] = g.N; g.N += c.second.first; }
    for (auto &x : kv.second.xs) { g.x_off[x.first] = g.K; g.K += x.second; }
    if (g.M > INT32_MAX || g.N > INT32_MAX || g.K > INT32_MAX) { err = "sector too large"; return YTN_E_UNSUPPORTED; }
    geo.push_back(std::move(g));
    sbs.push_back(&kv.second);
  }

  // Operand layouts: choose, per operand, the sector-matrix orientation in which
  // most gathered elements keep their source-contiguous dimension innermost.
  auto count_contig = [&](const Tensor &T, const std::vector<int> &first, const std::vector<int> &second) {
    // elements whose innermost destination dim is the source's innermost leg
    double same = 0, total = 0;
    for (int64_t b = 0; b < T.nblocks; b++) {
      const double e = (double)T.elems(b);
      total += e;
      int last_src = -1;
      for (int i = T.rank - 1; i >= 0; i--)
        if (T.dim(b, i) != 1) { last_src = i; break; }
      int last_dst = -1;
      for (int i = (int)second.size() - 1; i >= 0 && last_dst < 0; i--)
        if (T.dim(b, second[i]) != 1) last_dst = second[i];
      for (int i = (int)first.size() - 1; i >= 0 && last_dst < 0; i--)
        if (T.dim(b, first[i]) != 1) last_dst = first[i];
      if (last_src == last_dst) same += e;
    }
    return same;
  };
  {
    const double a_mk = count_contig(A, freeA, axa), a_km = count_contig(A, axa, freeA);
    const double b_nk = count_contig(B, freeB, axb), b_kn = count_contig(B, axb, freeB);
    p->a_kmajor = a_mk >= a_km;
    p->b_kmajor = b_nk > b_kn;
  }

  // Workspace offsets of the sector matrices (256-byte aligned per sector).
  auto align32 = [](int64_t e) { return (e + 31) / 32 * 32; };
  p->sectors.clear();
  p->sectors_dev.clear();
  int64_t ao = 0, bo = 0, co = 0;
  int64_t a_cov = 0, b_cov = 0;
  p->max_m = p->max_n = p->max_k = 0;
  for (auto &g : geo) {
    HostSector h;   // the GEMM's (real, possibly doubled) geometry
    h.M = ca * g.M; h.N = cb * g.N; h.K = g.K;
    if (h.M > INT32_MAX || h.N > INT32_MAX) { err = "sector too large"; return YTN_E_UNSUPPORTED; }
    h.a_off = ao; h.b_off = bo; h.c_off = co;
    ao += align32(h.M * h.K);
    bo += align32(h.K * h.N);
    co += align32(h.M * h.N);
    p->sectors.push_back(h);
    SectorDev d{};
    d.a_off = h.a_off; d.b_off = h.b_off; d.c_off = h.c_off;
    d.M = (int32_t)h.M; d.N = (int32_t)h.N; d.K = (int32_t)h.K;
    d.a_kmajor = p->a_kmajor; d.b_kmajor = p->b_kmajor;
    p->sectors_dev.push_back(d);
    p->max_m = std::max(p->max_m, h.M);
    p->max_n = std::max(p->max_n, h.N);
    p->max_k = std::max(p->max_k, h.K);
  }
  p->a_elems = ao;
  p->b_elems = bo;
  p->c_elems = co;

  p->jobs.clear();
  p->items.clear();
  p->moved = 0;
  // Where each block lands in its sector matrix, for the fused split: rows
  // [roff, roff + rlen) and K [koff, koff + klen) of the operand (A_q, or B_q
  // transposed), with the block's free and contracted dims and their strides.
  std::vector<SegSource> seg_src[2];
  std::vector<size_t> sec_jobs[2];   // first job of each sector, per operand
  // Gather A: block (I, x) -> A_q[row_off(I) + i, x_off(x) + k].
  // isA: gather A (free part = rows M) else B (free part = columns N).
  auto gather = [&](const Tensor &T, const std::vector<int> &freeL, const std::vector<int> &conL,
                    bool isA, bool kmajor, int64_t &covered) -> ytn_status {
    for (size_t si = 0; si < geo.size(); si++) {
      const SG &g = geo[si];
      const HostSector &h = p->sectors[si];
      sec_jobs[isA ? 0 : 1].push_back(p->jobs.size());
      for (auto &xk : g.x_off) {
        const auto &blist = isA ? Ax[xk.first] : Bx[xk.first];
        for (int64_t b : blist) {
          Key fk = sub_charges(T, b, freeL);
          const auto &offmap = isA ? g.row_off : g.col_off;
          auto it = offmap.find(fk);
          if (it == offmap.end()) continue;
          const int64_t foff = it->second, xoff = xk.second;
          const int cw = isA ? ca : cb;         // 2: complex operand
          const int64_t F = isA ? h.M : h.N;    // free extent of the (doubled) sector matrix
          const int64_t base = isA ? h.a_off : h.b_off;
          auto st = block_strides(T, b);
          // strides of the free and contracted sub-indices inside their fused index
          std::vector<Dim> dims;
          std::vector<int64_t> fstr(freeL.size()), cstr(conL.size());
          int64_t acc = 1;
          for (int i = (int)freeL.size() - 1; i >= 0; i--) { fstr[i] = acc; acc *= T.dim(b, freeL[i]); }
          acc = 1;
          for (int i = (int)conL.size() - 1; i >= 0; i--) { cstr[i] = acc; acc *= T.dim(b, conL[i]); }
          // kmajor: matrix is (free rows) x (K cols), ld = K; else (K rows) x (free cols), ld = F.
          const int64_t ldk = kmajor ? g.K : F;
          int64_t dst_off;
          if (kmajor) {
            for (size_t i = 0; i < freeL.size(); i++) dims.push_back({T.dim(b, freeL[i]), st[freeL[i]], fstr[i] * ldk});
            for (size_t i = 0; i < conL.size(); i++) dims.push_back({T.dim(b, conL[i]), st[conL[i]], cstr[i]});
            dst_off = base + foff * ldk + xoff;
          } else {
            for (size_t i = 0; i < conL.size(); i++) dims.push_back({T.dim(b, conL[i]), st[conL[i]], cstr[i] * ldk});
            for (size_t i = 0; i < freeL.size(); i++) dims.push_back({T.dim(b, freeL[i]), st[freeL[i]], fstr[i]});
            dst_off = base + xoff * ldk + foff;
          }
          int64_t src_off = T.off[b];
          for (int comp = 0; comp < cw; comp++) {
            SegSource ss;
            ss.sector = (int64_t)si;
            ss.roff = foff + comp * (isA ? g.M : g.N);
            ss.koff = xoff;
            ss.boff = cw * src_off + comp;
            ss.rlen = 1;
            for (size_t i = 0; i < freeL.size(); i++) {
              ss.fext.push_back(T.dim(b, freeL[i]));
              ss.fst.push_back(cw * st[freeL[i]]);
              ss.rlen *= T.dim(b, freeL[i]);
            }
            ss.klen = 1;
            for (size_t i = 0; i < conL.size(); i++) {
              ss.kext.push_back(T.dim(b, conL[i]));
              ss.kst.push_back(cw * st[conL[i]]);
              ss.klen *= T.dim(b, conL[i]);
            }
            seg_src[isA ? 0 : 1].push_back(std::move(ss));
          }
          if (cw == 2) {
            // interleaved (re, im) source: element strides double; the component
            // selects the row block (A) or column block (B) of the sector matrix
            for (auto &d : dims) d.sst *= 2;
            src_off *= 2;
            const int64_t half = isA ? g.M : g.N;
            dims.push_back({2, 1, kmajor ? half * g.K : half});
          }
          ytn_status s = add_copy(p, dims, src_off, dst_off, err);
          if (s != YTN_OK) return s;
          covered += T.elems(b);
          p->moved += T.elems(b);
        }
      }
    }
    return YTN_OK;
  };
  // Work items per sector (an item never spans two sectors), so that the FP64
  // fallback of the split path can gather the sectors it recomputes alone.
  p->sec_gather_items.assign(geo.size(), {0, 0, 0, 0});
  auto items_per_sector = [&](int which, size_t jend, int64_t base) {
    const auto &sj = sec_jobs[which];
    for (size_t si = 0; si < sj.size(); si++) {
      const size_t a = sj[si], b = si + 1 < sj.size() ? sj[si + 1] : jend;
      p->sec_gather_items[si][2 * which] = (int64_t)p->items.size() - base;
      make_items(p, a, b);
      p->sec_gather_items[si][2 * which + 1] = (int64_t)p->items.size() - base;
    }
  };
  size_t j0 = p->jobs.size();
  ytn_status s = gather(A, freeA, axa, true, p->a_kmajor, a_cov);
  if (s != YTN_OK) return s;
  size_t j1 = p->jobs.size();
  p->items_a_begin = (int64_t)p->items.size();
  (void)j0;
  items_per_sector(0, j1, p->items_a_begin);
  p->items_a_end = (int64_t)p->items.size();
  s = gather(B, freeB, axb, false, p->b_kmajor, b_cov);
  if (s != YTN_OK) return s;
  size_t j2 = p->jobs.size();
  p->items_b_begin = (int64_t)p->items.size();
  items_per_sector(1, j2, p->items_b_begin);
  p->items_b_end = (int64_t)p->items.size();
  int64_t a_need = 0, b_need = 0;
  for (auto &g : geo) { a_need += g.M * g.K; b_need += g.K * g.N; }
  p->zero_a = a_cov < a_need;
  p->zero_b = b_cov < b_need;

  // Output blocks: (I, J) exists when some x has both A(I, x) and B(x, J).
  std::vector<OutBlock> outb;
  struct Src { int64_t sector; int64_t roff, coff; int64_t nI, nJ; int64_t a_blk, b_blk; };
  std::vector<Src> srcs;
  for (size_t si = 0; si < geo.size(); si++) {
    const SG &g = geo[si];
    const SB &sb = *sbs[si];
    // x index per sector
    std::map<Key, int> xidx;
    for (auto &x : g.x_off) xidx.emplace(x.first, (int)xidx.size());
    const int nw = ((int)xidx.size() + 63) / 64;
    std::map<Key, std::vector<uint64_t>> rowx, colx;
    for (auto &x : g.x_off) {
      const int xi = xidx[x.first];
      for (int64_t a : Ax[x.first]) {
        auto &v = rowx[sub_charges(A, a, freeA)];
        v.resize(nw, 0);
        v[xi / 64] |= 1ull << (xi % 64);
      }
      for (int64_t b : Bx[x.first]) {
        auto &v = colx[sub_charges(B, b, freeB)];
        v.resize(nw, 0);
        v[xi / 64] |= 1ull << (xi % 64);
      }
    }
    for (auto &r : sb.rows) {
      const auto &rv = rowx[r.first];
      for (auto &c : sb.cols) {
        const auto &cv = colx[c.first];
        bool hit = false;
        for (int w = 0; w < nw && !hit; w++) hit = (rv[w] & cv[w]) != 0;
        if (!hit) continue;
        OutBlock ob;
        ob.key = r.first;
        ob.key.insert(ob.key.end(), c.first.begin(), c.first.end());
        for (int l : freeA) ob.D.push_back(A.dim(r.second.second, l));
        for (int l : freeB) ob.D.push_back(B.dim(c.second.second, l));
        ob.id = (int64_t)srcs.size();
        outb.push_back(ob);
        srcs.push_back({(int64_t)si, g.row_off.at(r.first), g.col_off.at(c.first), r.second.first,
                        c.second.first, r.second.second, c.second.second});
      }
    }
  }
  std::vector<int64_t> off_of_id;
  finalize_out(C, outb, off_of_id);
  // Scatter C: block (I, J) = C_q[row_off(I) + i, col_off(J) + j], row-major per leg.
  p->cs_jobs.clear();
  for (size_t id = 0; id < srcs.size() && ca * cb > 1; id++) {
    // complex product: combine the quadrants of the doubled C_q
    const Src &sr = srcs[id];
    const HostSector &h = p->sectors[sr.sector];
    const SG &g = geo[sr.sector];
    std::vector<int64_t> cd;
    for (int l : freeA) cd.push_back(A.dim(sr.a_blk, l));
    for (int l : freeB) cd.push_back(B.dim(sr.b_blk, l));
    if ((int)cd.size() > kMaxCopyDims) { err = "output block with more than 8 dims"; return YTN_E_UNSUPPORTED; }
    CScatterJob J{};
    J.src = h.c_off + sr.roff * h.N + sr.coff;
    J.dst = off_of_id[id];
    J.q01 = cb == 2 ? g.N : -1;
    J.q10 = ca == 2 ? g.M * h.N : -1;
    J.q11 = (ca == 2 && cb == 2) ? g.M * h.N + g.N : -1;
    J.nd = (int32_t)cd.size();
    int64_t acc = 1;
    for (int i = (int)freeA.size() - 1; i >= 0; i--) { J.sstr[i] = acc * h.N; acc *= cd[i]; }
    acc = 1;
    for (int i = (int)cd.size() - 1; i >= (int)freeA.size(); i--) { J.sstr[i] = acc; acc *= cd[i]; }
    int64_t n = 1;
    for (size_t i = 0; i < cd.size(); i++) {
      J.ext[i] = (int32_t)cd[i];
      n *= cd[i];
    }
    if (n > INT32_MAX) { err = "output block too large"; return YTN_E_UNSUPPORTED; }
    J.n = (int32_t)n;
    p->cs_jobs.push_back(J);
    p->moved += n;
  }
  for (size_t id = 0; id < srcs.size() && ca * cb == 1; id++) {
    const Src &sr = srcs[id];
    const HostSector &h = p->sectors[sr.sector];
    std::vector<Dim> dims;
    std::vector<int64_t> ds(C.rank);
    // destination: the C block, row-major over its legs
    std::vector<int64_t> cd;
    for (int l : freeA) cd.push_back(A.dim(sr.a_blk, l));
    for (int l : freeB) cd.push_back(B.dim(sr.b_blk, l));
    int64_t acc = 1;
    for (int i = C.rank - 1; i >= 0; i--) { ds[i] = acc; acc *= cd[i]; }
    const int64_t nblk = acc;
    // source: inside I the legs are row-major, times ldc = N; inside J row-major
    std::vector<int64_t> ss(C.rank);
    acc = 1;
    for (int i = (int)freeA.size() - 1; i >= 0; i--) { ss[i] = acc * h.N; acc *= cd[i]; }
    acc = 1;
    for (int i = C.rank - 1; i >= (int)freeA.size(); i--) { ss[i] = acc; acc *= cd[i]; }
    for (int i = 0; i < C.rank; i++) dims.push_back({cd[i], ss[i], ds[i]});
    s = add_copy(p, dims, h.c_off + sr.roff * h.N + sr.coff, off_of_id[id], err);
    if (s != YTN_OK) return s;
    p->moved += nblk;
  }
  size_t j3 = p->jobs.size();
  p->items_c_begin = (int64_t)p->items.size();
  make_items(p, j2, j3);
  p->items_c_end = (int64_t)p->items.size();

  // Grouped-GEMM tiles, largest K first. The tile edge is chosen per sector from
  // its size: 32 when 32 x 32 tiles cover the sector with at most 60% of the
  // padded area of 64 x 64 tiles (small or thin M, N), else 64.
  p->tiles.clear();
  for (size_t si = 0; si < geo.size(); si++) {
    const int64_t M = p->sectors[si].M, N = p->sectors[si].N;
    const int64_t a64 = ((M + 63) / 64) * ((N + 63) / 64) * 4096, a32 = ((M + 31) / 32) * ((N + 31) / 32) * 1024;
    const int T = 10 * a32 <= 6 * a64 ? 32 : 64;
    const int64_t mt = (M + T - 1) / T, nt = (N + T - 1) / T;
    for (int64_t i = 0; i < mt; i++)
      for (int64_t j = 0; j < nt; j++) p->tiles.push_back({(int32_t)si, (int32_t)i, (int32_t)j, T});
  }
  std::stable_sort(p->tiles.begin(), p->tiles.end(), [&](const GemmTile &x, const GemmTile &y) {
    return geo[x.sector].K > geo[y.sector].K;
  });
  plan_split_tables(p, seg_src);
  p->kind = Kind::Tensordot;
  p->a_size = A.size;
  p->b_size = B.size;
  return YTN_OK;
}

// Tables of the split-precision path: per sector, the slice blocks and exponents
// of A (rows M) and B (rows N), the exponent / slicing work items and the
// 128 x 128 output tiles (sectors by decreasing K; inside a sector, groups of 8
// row tiles with the column tiles innermost, so that CTAs running at the same time
// share operand slices in L2). When every block's dims fit kFusedDims per side,
// also the fused path's items and segments (slices straight from the blocks).
void plan_split_tables(ytn_plan_t *p, std::vector<SegSource> *src) {
  p->sp_ops.clear();
  p->sp_exp_items.clear();
  p->sp_slice_items.clear();
  p->sp_sectors.clear();
  p->sp_tiles.clear();
  p->sp_tiles_mix.clear();
  p->sp_fitems.clear();
  p->sp_segs.clear();
  p->sp_pipe_tile_end.clear();
  p->sp_pipe_item_end.clear();
  int64_t sa = 0, sb = 0, ea = 0, eb = 0;
  const int64_t nsec = (int64_t)p->sectors.size();
  for (int64_t q = 0; q < nsec; q++) {
    const HostSector &h = p->sectors[q];
    const int64_t tm = (h.M + kSplitBM - 1) / kSplitBM, tn = (h.N + kSplitBM - 1) / kSplitBM;
    const int64_t ks = (h.K + kSplitBK - 1) / kSplitBK;
    SplitSector s{};
    s.sa_off = sa;
    s.sb_off = sb;
    s.ea_off = ea;
    s.eb_off = eb;
    s.c_off = h.c_off;
    s.M = (int32_t)h.M;
    s.N = (int32_t)h.N;
    s.K = (int32_t)h.K;
    s.ks = (int32_t)ks;
    if ((size_t)q < p->sec_gather_items.size()) {
      s.ga0 = (int32_t)p->sec_gather_items[q][0];
      s.ga1 = (int32_t)p->sec_gather_items[q][1];
      s.gb0 = (int32_t)p->sec_gather_items[q][2];
      s.gb1 = (int32_t)p->sec_gather_items[q][3];
    }
    p->sp_sectors.push_back(s);
    SplitOperand oa{h.a_off, ea, sa, (int32_t)h.M, (int32_t)h.K, (int32_t)ks, p->a_kmajor ? 1 : 0};
    SplitOperand ob{h.b_off, eb, sb, (int32_t)h.N, (int32_t)h.K, (int32_t)ks, p->b_kmajor ? 1 : 0};
    const int32_t ia = (int32_t)p->sp_ops.size();
    p->sp_ops.push_back(oa);
    p->sp_ops.push_back(ob);
    for (int which = 0; which < 2; which++) {
      const int64_t tiles = which == 0 ? tm : tn;
      for (int64_t rt = 0; rt < tiles; rt++) {
        for (int64_t k0 = 0; k0 < ks; k0 += 8)   // row maxima per 256 of K, combined by atomicMax
          p->sp_exp_items.push_back({ia + which, (int32_t)rt, (int32_t)k0, (int32_t)std::min<int64_t>(8, ks - k0)});
        for (int64_t k0 = 0; k0 < ks; k0 += 8)
          p->sp_slice_items.push_back({ia + which, (int32_t)rt, (int32_t)k0, (int32_t)std::min<int64_t>(8, ks - k0)});
      }
    }
    sa += tm * ks * kBlockBytes;
    sb += tn * ks * kBlockBytes;
    ea += tm * kSplitBM;
    eb += tn * kSplitBM;
  }
  p->sp_sa_bytes = sa;
  p->sp_sb_bytes = sb;
  p->sp_ea = ea;
  p->sp_eb = eb;
  std::vector<int64_t> order(nsec);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t x, int64_t y) { return p->sectors[x].K > p->sectors[y].K; });
  // Tile lists: all 128 wide, and the same with the last column tile of a sector 64
  // wide where the sector's N ends in its first half (N mod 128 in 1..64: half of the
  // padded products of that tile saved). The first split call on a plan times both
  // when they differ and keeps the faster.
  p->sp_tiles_mix.clear();
  bool any_narrow = false;
  for (int64_t q : order) {
    const HostSector &h = p->sectors[q];
    const int64_t tm = (h.M + kSplitBM - 1) / kSplitBM, tn = (h.N + kSplitBM - 1) / kSplitBM;
    const bool tail_narrow = h.N % kSplitBM != 0 && h.N % kSplitBM <= kSplitBM / 2;
    any_narrow = any_narrow || tail_narrow;
    for (int64_t g0 = 0; g0 < tm; g0 += 8)
      for (int64_t n = 0; n < tn; n++)
        for (int64_t m = g0; m < std::min<int64_t>(g0 + 8, tm); m++) {
          p->sp_tiles.push_back({(int32_t)q, (int32_t)m, (int32_t)n, kSplitBM});
          if (tail_narrow && n == tn - 1)
            p->sp_tiles_mix.push_back({(int32_t)q, (int32_t)m, (int32_t)(2 * n), kSplitBM / 2});
          else
            p->sp_tiles_mix.push_back({(int32_t)q, (int32_t)m, (int32_t)n, kSplitBM});
        }
  }
  if (!any_narrow) p->sp_tiles_mix.clear();

  // Fused path: items of 32 rows x 128 of K per operand, each with the parts of
  // the blocks inside it. Unit dims are dropped and neighbouring dims that are
  // contiguous in the block merged; a block with more than kFusedDims dims on
  // either side, or spanning more than 2^30 elements, leaves the fused path off
  // (the staged path gathers first). Three per side cover the contractions of the
  // CTM workloads (their free and contracted legs merge to one or two dims each).
  p->sp_fused = false;
  if (!src) return;
  auto squeeze = [](std::vector<int64_t> &ext, std::vector<int64_t> &st) {
    std::vector<int64_t> e2, s2;
    for (size_t i = 0; i < ext.size(); i++) {
      if (ext[i] == 1) continue;
      if (!e2.empty() && s2.back() == st[i] * ext[i]) {
        e2.back() *= ext[i];
        s2.back() = st[i];
      } else {
        e2.push_back(ext[i]);
        s2.push_back(st[i]);
      }
    }
    ext.swap(e2);
    st.swap(s2);
  };
  for (int w = 0; w < 2; w++)
    for (SegSource &ss : src[w]) {
      squeeze(ss.fext, ss.fst);
      squeeze(ss.kext, ss.kst);
      if (ss.fext.size() > (size_t)kFusedDims || ss.kext.size() > (size_t)kFusedDims) return;
      int64_t span = 0;   // largest offset of an element inside the block
      for (size_t i = 0; i < ss.fext.size(); i++) span += (ss.fext[i] - 1) * ss.fst[i];
      for (size_t i = 0; i < ss.kext.size(); i++) span += (ss.kext[i] - 1) * ss.kst[i];
      if (span > INT32_MAX / 2) return;   // 32-bit offsets, one step past the end included
    }
  // items: per operand (A of sector q is op 2q, B op 2q + 1), 32-row quarters of
  // the 128-row tiles x 128 of K
  std::vector<int64_t> item_base(p->sp_ops.size() + 1, 0);
  auto nkq = [](const SplitOperand &op) { return ((int64_t)op.ks * kSplitBK + kItemK - 1) / kItemK; };
  auto nrq = [](const SplitOperand &op) { return (int64_t)((op.rows + kSplitBM - 1) / kSplitBM) * (kSplitBM / kItemRows); };
  for (size_t o = 0; o < p->sp_ops.size(); o++) item_base[o + 1] = item_base[o] + nrq(p->sp_ops[o]) * nkq(p->sp_ops[o]);
  const int64_t nitems = item_base.back();
  std::vector<std::vector<SliceSeg>> per_item(nitems);
  std::vector<int64_t> covered(nitems, 0);
  for (int w = 0; w < 2; w++)
    for (const SegSource &ss : src[w]) {
      const int64_t o = 2 * ss.sector + w;
      const SplitOperand &op = p->sp_ops[o];
      if (ss.rlen <= 0 || ss.klen <= 0) continue;
      for (int64_t hr = ss.roff / kItemRows; hr <= (ss.roff + ss.rlen - 1) / kItemRows; hr++)
        for (int64_t c = ss.koff / kItemK; c <= (ss.koff + ss.klen - 1) / kItemK; c++) {
          const int64_t ra = std::max(ss.roff, hr * kItemRows), rb = std::min(ss.roff + ss.rlen, hr * kItemRows + kItemRows);
          const int64_t ka = std::max(ss.koff, c * kItemK), kb = std::min(ss.koff + ss.klen, c * kItemK + kItemK);
          SliceSeg g{};
          g.boff = ss.boff;
          g.nf = (uint8_t)ss.fext.size();
          g.nk = (uint8_t)ss.kext.size();
          for (size_t i = 0; i < ss.fext.size(); i++) {
            g.fext[i] = (int32_t)ss.fext[i];
            g.fst[i] = ss.fst[i];
          }
          for (size_t i = 0; i < ss.kext.size(); i++) {
            g.kext[i] = (int32_t)ss.kext[i];
            g.kst[i] = ss.kst[i];
          }
          g.ibase = (int32_t)(ra - ss.roff);
          g.kbase = (int32_t)(ka - ss.koff);
          g.r0 = (int16_t)(ra - hr * kItemRows);
          g.r1 = (int16_t)(rb - hr * kItemRows);
          g.k0 = (int16_t)(ka - c * kItemK);
          g.k1 = (int16_t)(kb - c * kItemK);
          // rows fastest when the block's innermost free stride is below its
          // innermost contracted stride (consecutive rows are nearer in memory)
          const int64_t fs = ss.fst.empty() ? INT64_MAX : ss.fst.back();
          const int64_t kst = ss.kst.empty() ? INT64_MAX : ss.kst.back();
          g.rfast = fs < kst ? 1 : 0;
          const int64_t it = item_base[o] + hr * nkq(op) + c;
          per_item[it].push_back(g);
          covered[it] += (rb - ra) * (kb - ka);
        }
    }
  // items in the GEMM's sector order (decreasing K), A's before B's per sector, so
  // that a run of sectors in that order is a run of items (pipelined slicing)
  std::vector<int64_t> sec_item_end;
  for (int64_t oq = 0; oq < 2 * nsec; oq++) {
    const size_t o = (size_t)(2 * order[oq / 2] + oq % 2);
    const SplitOperand &op = p->sp_ops[o];
    for (int64_t hr = 0; hr < nrq(op); hr++)
      for (int64_t c = 0; c < nkq(op); c++) {
        const int64_t it = item_base[o] + hr * nkq(op) + c;
        SliceItem si{};
        si.op = (int32_t)o;
        si.rt = (int32_t)(hr / (kSplitBM / kItemRows));
        si.quarter = (int32_t)(hr % (kSplitBM / kItemRows));
        si.kq = (int32_t)c;
        si.seg0 = (int32_t)p->sp_segs.size();
        si.nseg = (int32_t)per_item[it].size();
        const int64_t kc = std::min<int64_t>(kItemK, (int64_t)op.ks * kSplitBK - c * kItemK);
        si.full = covered[it] == kItemRows * kc ? 1 : 0;
        int32_t cost = 0;   // warp-wide copy steps (at most 32 rows x 128 of K)
        for (SliceSeg &g : per_item[it]) {
          g.cost0 = cost;
          const int32_t nr = g.r1 - g.r0, nk = g.k1 - g.k0;
          cost += g.rfast ? nk : nr * ((nk + 31) / 32);
        }
        si.cost = cost;
        p->sp_fitems.push_back(si);
        p->sp_segs.insert(p->sp_segs.end(), per_item[it].begin(), per_item[it].end());
        if (p->sp_segs.size() > (size_t)INT32_MAX) {
          p->sp_fitems.clear();
          p->sp_segs.clear();
          return;
        }
      }
    if (oq % 2 == 1) sec_item_end.push_back((int64_t)p->sp_fitems.size());
  }
  p->sp_fused = true;

  // Pipeline groups: runs of sectors in the GEMM's order of about an eighth of the
  // useful FLOPs each, every group holding at least two waves of 128-wide tiles
  // (one CTA per SM), so that each group's GEMM launch fills the GPU; the last run
  // joins its predecessor when it is shorter. Fewer than two groups: no pipeline.
  const int64_t min_tiles = 2 * (int64_t)std::max(1, p->ctx ? p->ctx->num_sms : 0);
  double total = 0.0;
  for (int64_t q : order) total += 2.0 * p->sectors[q].M * p->sectors[q].N * p->sectors[q].K;
  int64_t tile_end = 0, gt = 0;
  double gf = 0.0;
  for (int64_t oi = 0; oi < nsec; oi++) {
    const HostSector &h = p->sectors[order[oi]];
    const int64_t nt = ((h.M + kSplitBM - 1) / kSplitBM) * ((h.N + kSplitBM - 1) / kSplitBM);
    tile_end += nt;
    gt += nt;
    gf += 2.0 * h.M * h.N * h.K;
    const bool last = oi == nsec - 1;
    if ((gf >= total / kPipeGroups && gt >= min_tiles) || last) {
      if (last && gt < min_tiles && !p->sp_pipe_tile_end.empty()) {
        p->sp_pipe_tile_end.back() = tile_end;
        p->sp_pipe_item_end.back() = sec_item_end[oi];
      } else {
        p->sp_pipe_tile_end.push_back(tile_end);
        p->sp_pipe_item_end.push_back(sec_item_end[oi]);
      }
      gt = 0;
      gf = 0.0;
    }
  }
  if (p->sp_pipe_tile_end.size() < 2 || p->ctx == nullptr || p->ctx->device < 0) {
    p->sp_pipe_tile_end.clear();
    p->sp_pipe_item_end.clear();
  }
}

// ---------------------------------------------------------------------------
// Fuse
// ---------------------------------------------------------------------------

ytn_status plan_fuse(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size,
                     const int *order, std::string &err) {
  if (ngroups < 1 || ngroups > YTN_MAX_RANK) { err = "ngroups out of range"; return YTN_E_INVALID; }
  std::vector<std::vector<int>> groups;
  std::vector<int> seen(A.rank, 0);
  int pos = 0;
  for (int g = 0; g < ngroups; g++) {
    if (group_size[g] < 1 || pos + group_size[g] > A.rank) { err = "bad group sizes"; return YTN_E_INVALID; }
    std::vector<int> grp;
    for (int i = 0; i < group_size[g]; i++) {
      const int l = order[pos++];
      if (l < 0 || l >= A.rank || seen[l]) { err = "fusion groups must list every leg once"; return YTN_E_INVALID; }
      seen[l] = 1;
      grp.push_back(l);
    }
    groups.push_back(grp);
  }
  if (pos != A.rank) { err = "fusion groups must list every leg once"; return YTN_E_INVALID; }
  for (auto &g : groups)
    if (g.size() > 1)
      for (int l : g)
        if (A.fus[l]) { err = "fusing an already fused leg"; return YTN_E_UNSUPPORTED; }
  const int nsym = A.nsym;
  const int G = ngroups;
  // fused charge of block b for group g: nu = s_r sum_i s_i rho_i (s_r: first leg)
  auto nu_of = [&](int64_t b, const std::vector<int> &g) {
    Key nu(nsym, 0);
    for (int c = 0; c < nsym; c++) {
      int64_t tot = 0;
      for (int l : g) tot += (int64_t)A.sig[l] * A.charge(b, l)[c];
      nu[c] = reduce((int64_t)A.sig[g[0]] * tot, A.mod[c]);
    }
    return nu;
  };
  // Records: per group, nu -> ascending constituent tuples with dims (lazy).
  std::vector<std::map<Key, std::map<Key, std::vector<int64_t>>>> rec(G);
  for (int g = 0; g < G; g++) {
    if (groups[g].size() < 2) continue;
    for (int64_t b = 0; b < A.nblocks; b++) {
      Key ch = sub_charges(A, b, groups[g]);
      std::vector<int64_t> d;
      for (int l : groups[g]) d.push_back(A.dim(b, l));
      rec[g][nu_of(b, groups[g])].emplace(ch, d);
    }
  }
  // offsets of each constituent tuple inside its fused sector, and D_nu
  std::vector<std::map<Key, std::map<Key, int64_t>>> suboff(G);
  std::vector<std::map<Key, int64_t>> dnu(G);
  for (int g = 0; g < G; g++)
    for (auto &kv : rec[g]) {
      int64_t acc = 0;
      for (auto &e : kv.second) {
        suboff[g][kv.first][e.first] = acc;
        int64_t sz = 1;
        for (auto d : e.second) sz *= d;
        acc += sz;
      }
      dnu[g][kv.first] = acc;
    }
  Tensor &C = p->out;
  C = Tensor();
  C.dtype = A.dtype;
  p->cw = A.dtype == YTN_COMPLEX128 ? 2 : 1;
  C.nsym = nsym;
  std::memcpy(C.mod, A.mod, sizeof(C.mod));
  std::memcpy(C.n, A.n, sizeof(C.n));
  C.rank = G;
  for (int g = 0; g < G; g++) {
    C.sig[g] = A.sig[groups[g][0]];
    if (groups[g].size() == 1) {
      copy_fusion(A.fus[groups[g][0]].get(), C.fus[g]);
      continue;
    }
    auto F = std::make_shared<Fusion>();
    F->nlegs = (int)groups[g].size();
    for (int j = 0; j < F->nlegs; j++) F->sig[j] = A.sig[groups[g][j]];
    for (auto &kv : rec[g])
      for (auto &e : kv.second) {
        F->nu.insert(F->nu.end(), kv.first.begin(), kv.first.end());
        F->t.insert(F->t.end(), e.first.begin(), e.first.end());
        F->D.insert(F->D.end(), e.second.begin(), e.second.end());
        F->nentries++;
      }
    C.fus[g] = F;
  }
  // New blocks.
  std::map<Key, int64_t> newid;
  std::vector<OutBlock> outb;
  std::vector<int64_t> blk_new(A.nblocks);
  for (int64_t b = 0; b < A.nblocks; b++) {
    Key k;
    std::vector<int64_t> D;
    for (int g = 0; g < G; g++) {
      if (groups[g].size() == 1) {
        const int32_t *q = A.charge(b, groups[g][0]);
        k.insert(k.end(), q, q + nsym);
        D.push_back(A.dim(b, groups[g][0]));
      } else {
        Key nu = nu_of(b, groups[g]);
        k.insert(k.end(), nu.begin(), nu.end());
        D.push_back(dnu[g][nu]);
      }
    }
    auto it = newid.find(k);
    if (it == newid.end()) {
      const int64_t id = (int64_t)outb.size();
      newid[k] = id;
      outb.push_back({k, D, id});
      blk_new[b] = id;
    } else {
      blk_new[b] = it->second;
    }
  }
  std::vector<OutBlock> sorted = outb;
  std::vector<int64_t> off_of_id;
  finalize_out(C, sorted, off_of_id);
  // Copy jobs: old block, legs in group order -> its sub-box of the new block.
  p->jobs.clear();
  p->items.clear();
  p->moved = 0;
  for (int64_t b = 0; b < A.nblocks; b++) {
    const OutBlock &ob = outb[blk_new[b]];
    std::vector<int64_t> nst(G);
    int64_t acc = 1;
    for (int g = G - 1; g >= 0; g--) { nst[g] = acc; acc *= ob.D[g]; }
    auto st = block_strides(A, b);
    std::vector<Dim> dims;
    int64_t dst_off = off_of_id[ob.id];
    for (int g = 0; g < G; g++) {
      const auto &grp = groups[g];
      int64_t in = 1;
      std::vector<int64_t> gs(grp.size());
      for (int i = (int)grp.size() - 1; i >= 0; i--) { gs[i] = in; in *= A.dim(b, grp[i]); }
      for (size_t i = 0; i < grp.size(); i++) dims.push_back({A.dim(b, grp[i]), st[grp[i]], gs[i] * nst[g]});
      if (grp.size() > 1) {
        Key nu = nu_of(b, grp);
        dst_off += suboff[g][nu][sub_charges(A, b, grp)] * nst[g];
      }
    }
    ytn_status s = add_copy(p, dims, A.off[b], dst_off, err);
    if (s != YTN_OK) return s;
    p->moved += A.elems(b);
  }
  make_items(p, 0, p->jobs.size());
  p->items_a_begin = 0;
  p->items_a_end = (int64_t)p->items.size();
  p->zero_out = p->moved < C.size;
  p->kind = Kind::Fuse;
  p->a_size = A.size;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Unfuse
// ---------------------------------------------------------------------------

ytn_status plan_unfuse(ytn_plan_t *p, const Tensor &A, int naxes, const int *axes_in, std::string &err) {
  std::vector<int> isun(A.rank, 0);
  if (naxes < 1) { err = "no legs to unfuse"; return YTN_E_INVALID; }
  for (int k = 0; k < naxes; k++) {
    const int a = axes_in[k];
    if (a < 0 || a >= A.rank || !A.fus[a] || isun[a]) { err = "leg is not a fused leg"; return YTN_E_INVALID; }
    isun[a] = 1;
  }
  const int nsym = A.nsym;
  Tensor &C = p->out;
  C = Tensor();
  C.dtype = A.dtype;
  p->cw = A.dtype == YTN_COMPLEX128 ? 2 : 1;
  C.nsym = nsym;
  std::memcpy(C.mod, A.mod, sizeof(C.mod));
  std::memcpy(C.n, A.n, sizeof(C.n));
  int r = 0;
  for (int a = 0; a < A.rank; a++) {
    if (isun[a]) {
      for (int j = 0; j < A.fus[a]->nlegs; j++) {
        if (r >= YTN_MAX_RANK) { err = "output rank too large"; return YTN_E_UNSUPPORTED; }
        C.sig[r++] = A.fus[a]->sig[j];
      }
    } else {
      if (r >= YTN_MAX_RANK) { err = "output rank too large"; return YTN_E_UNSUPPORTED; }
      copy_fusion(A.fus[a].get(), C.fus[r]);
      C.sig[r++] = A.sig[a];
    }
  }
  C.rank = r;
  // per unfused leg: nu -> list of (charges, dims, offset)
  struct Ent { Key ch; std::vector<int64_t> d; int64_t off; };
  std::vector<std::map<Key, std::vector<Ent>>> ents(A.rank);
  for (int a = 0; a < A.rank; a++) {
    if (!isun[a]) continue;
    const Fusion &F = *A.fus[a];
    std::map<Key, int64_t> acc;
    for (int64_t e = 0; e < F.nentries; e++) {
      Key nu(&F.nu[e * nsym], &F.nu[e * nsym] + nsym);
      Ent en;
      en.ch.assign(&F.t[e * F.nlegs * nsym], &F.t[(e + 1) * F.nlegs * nsym]);
      en.d.assign(&F.D[e * F.nlegs], &F.D[(e + 1) * F.nlegs]);
      en.off = acc[nu];
      int64_t sz = 1;
      for (auto d : en.d) sz *= d;
      acc[nu] += sz;
      ents[a][nu].push_back(en);
    }
  }
  std::vector<OutBlock> outb;
  struct Src { int64_t blk; std::vector<const Ent *> pick; };
  std::vector<Src> srcs;
  for (int64_t b = 0; b < A.nblocks; b++) {
    std::vector<const std::vector<Ent> *> lists(A.rank, nullptr);
    int64_t combos = 1;
    for (int a = 0; a < A.rank; a++) {
      if (!isun[a]) continue;
      const int32_t *q = A.charge(b, a);
      auto it = ents[a].find(Key(q, q + nsym));
      if (it == ents[a].end()) { err = "fused block charge missing from its record"; return YTN_E_INVALID; }
      lists[a] = &it->second;
      combos *= (int64_t)it->second.size();
    }
    for (int64_t cidx = 0; cidx < combos; cidx++) {
      int64_t rem = cidx;
      std::vector<const Ent *> pick(A.rank, nullptr);
      for (int a = A.rank - 1; a >= 0; a--) {
        if (!isun[a]) continue;
        const int64_t n = (int64_t)lists[a]->size();
        pick[a] = &(*lists[a])[rem % n];
        rem /= n;
      }
      OutBlock ob;
      for (int a = 0; a < A.rank; a++) {
        if (isun[a]) {
          ob.key.insert(ob.key.end(), pick[a]->ch.begin(), pick[a]->ch.end());
          ob.D.insert(ob.D.end(), pick[a]->d.begin(), pick[a]->d.end());
        } else {
          const int32_t *q = A.charge(b, a);
          ob.key.insert(ob.key.end(), q, q + nsym);
          ob.D.push_back(A.dim(b, a));
        }
      }
      ob.id = (int64_t)srcs.size();
      outb.push_back(ob);
      srcs.push_back({b, pick});
    }
  }
  std::vector<OutBlock> sorted = outb;
  std::vector<int64_t> off_of_id;
  finalize_out(C, sorted, off_of_id);
  for (size_t i = 1; i < sorted.size(); i++)
    if (!(sorted[i - 1].key < sorted[i].key)) { err = "unfused blocks collide"; return YTN_E_INVALID; }
  p->jobs.clear();
  p->items.clear();
  p->moved = 0;
  for (size_t id = 0; id < srcs.size(); id++) {
    const Src &sr = srcs[id];
    const OutBlock &ob = outb[id];
    auto st = block_strides(A, sr.blk);
    std::vector<int64_t> dstr(ob.D.size());
    int64_t acc = 1;
    for (int i = (int)ob.D.size() - 1; i >= 0; i--) { dstr[i] = acc; acc *= ob.D[i]; }
    std::vector<Dim> dims;
    int64_t src_off = A.off[sr.blk];
    int r2 = 0;
    for (int a = 0; a < A.rank; a++) {
      if (isun[a]) {
        const Ent *e = sr.pick[a];
        src_off += e->off * st[a];
        int64_t in = 1;
        std::vector<int64_t> gs(e->d.size());
        for (int i = (int)e->d.size() - 1; i >= 0; i--) { gs[i] = in; in *= e->d[i]; }
        for (size_t i = 0; i < e->d.size(); i++, r2++) dims.push_back({e->d[i], gs[i] * st[a], dstr[r2]});
      } else {
        dims.push_back({A.dim(sr.blk, a), st[a], dstr[r2]});
        r2++;
      }
    }
    ytn_status s = add_copy(p, dims, src_off, off_of_id[ob.id], err);
    if (s != YTN_OK) return s;
    p->moved += acc;
  }
  make_items(p, 0, p->jobs.size());
  p->items_a_begin = 0;
  p->items_a_end = (int64_t)p->items.size();
  p->zero_out = false;
  p->kind = Kind::Unfuse;
  p->a_size = A.size;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Trace
// ---------------------------------------------------------------------------

ytn_status plan_trace(ytn_plan_t *p, const Tensor &A, int naxes, const int *ax1_in, const int *ax2_in,
                      std::string &err) {
  if (naxes < 1 || 2 * naxes > A.rank) { err = "bad number of traced pairs"; return YTN_E_INVALID; }
  std::vector<int> ax1(ax1_in, ax1_in + naxes), ax2(ax2_in, ax2_in + naxes);
  std::vector<int> used(A.rank, 0);
  for (int k = 0; k < naxes; k++) {
    for (int a : {ax1[k], ax2[k]}) {
      if (a < 0 || a >= A.rank || used[a]) { err = "trace axes must be distinct legs"; return YTN_E_INVALID; }
      used[a] = 1;
    }
  }
  for (int k = 0; k < naxes; k++) {
    ytn_status st = check_pair(A, ax1[k], A, ax2[k], err);
    if (st != YTN_OK) return st;
  }
  std::vector<int> rest;
  for (int i = 0; i < A.rank; i++)
    if (!used[i]) rest.push_back(i);
  if ((int)rest.size() > kMaxCopyDims || naxes > kMaxCopyDims) { err = "trace needs more than 8 dims"; return YTN_E_UNSUPPORTED; }
  const int nsym = A.nsym;
  const bool cplx = A.dtype == YTN_COMPLEX128;
  if (cplx && (int)rest.size() + 1 > kMaxCopyDims) { err = "trace needs more than 8 dims"; return YTN_E_UNSUPPORTED; }
  Tensor &C = p->out;
  C = Tensor();
  C.dtype = A.dtype;
  C.nsym = nsym;
  std::memcpy(C.mod, A.mod, sizeof(C.mod));
  std::memcpy(C.n, A.n, sizeof(C.n));
  C.rank = (int)rest.size();
  for (size_t i = 0; i < rest.size(); i++) {
    C.sig[i] = A.sig[rest[i]];
    copy_fusion(A.fus[rest[i]].get(), C.fus[i]);
  }
  std::map<Key, std::vector<int64_t>> contrib;   // out key -> contributing blocks (canonical order)
  std::map<Key, std::vector<int64_t>> outdims;
  for (int64_t b = 0; b < A.nblocks; b++) {
    bool ok = true;
    for (int k = 0; k < naxes && ok; k++) {
      const int32_t *q1 = A.charge(b, ax1[k]), *q2 = A.charge(b, ax2[k]);
      ok = std::equal(q1, q1 + nsym, q2);
      if (ok && A.dim(b, ax1[k]) != A.dim(b, ax2[k])) {
        err = "traced legs have different dimensions for one charge";
        return YTN_E_DIM_MISMATCH;
      }
    }
    if (!ok) continue;
    Key k = sub_charges(A, b, rest);
    contrib[k].push_back(b);
    std::vector<int64_t> d;
    for (int l : rest) d.push_back(A.dim(b, l));
    outdims[k] = d;
  }
  std::vector<OutBlock> outb;
  for (auto &kv : contrib) outb.push_back({kv.first, outdims[kv.first], (int64_t)outb.size()});
  std::vector<OutBlock> sorted = outb;
  std::vector<int64_t> off_of_id;
  finalize_out(C, sorted, off_of_id);
  p->tr_out.clear();
  p->tr_contrib.clear();
  int64_t id = 0;
  for (auto &kv : contrib) {
    TraceOut to{};
    to.dst_off = off_of_id[id];
    const auto &d = outdims[kv.first];
    int64_t nrest = 1;
    for (auto x : d) nrest *= x;
    if (nrest > INT32_MAX) { err = "trace output block too large"; return YTN_E_UNSUPPORTED; }
    to.nrest = (int32_t)nrest;
    to.nrd = (int32_t)d.size();
    for (size_t i = 0; i < d.size(); i++) to.rext[i] = (int32_t)d[i];
    to.first = (int32_t)p->tr_contrib.size();
    to.ncontrib = (int32_t)kv.second.size();
    // complex data: doubles instead of elements, the component an innermost rest dim
    const int w = cplx ? 2 : 1;
    if (cplx) {
      if (to.nrest > INT32_MAX / 2) { err = "trace output block too large"; return YTN_E_UNSUPPORTED; }
      to.dst_off *= 2;
      to.nrest *= 2;
      to.rext[to.nrd++] = 2;
    }
    for (int64_t b : kv.second) {
      TraceContrib tc{};
      tc.src_off = w * A.off[b];
      auto st = block_strides(A, b);
      for (size_t i = 0; i < rest.size(); i++) tc.rstr[i] = (int32_t)(w * st[rest[i]]);
      if (cplx) tc.rstr[rest.size()] = 1;
      tc.ndiag = naxes;
      for (int k = 0; k < naxes; k++) {
        tc.dext[k] = (int32_t)A.dim(b, ax1[k]);
        tc.dstr[k] = (int32_t)(w * (st[ax1[k]] + st[ax2[k]]));
      }
      p->tr_contrib.push_back(tc);
    }
    p->tr_out.push_back(to);
    id++;
  }
  p->kind = Kind::Trace;
  p->a_size = A.size;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Scalar product
// ---------------------------------------------------------------------------

static bool fusion_equal(const Fusion &a, const Fusion &b) {
  if (a.nlegs != b.nlegs || a.nentries != b.nentries) return false;
  for (int j = 0; j < a.nlegs; j++)
    if (a.sig[j] != b.sig[j]) return false;
  return a.nu == b.nu && a.t == b.t && a.D == b.D;
}

// <A, B>: the sum over the elements of the blocks present in both tensors of A's
// element times B's. The tensors must lie on the same legs: same symmetry, rank
// and signatures, one dimension per charge on each leg, identical fusion records.
ytn_status plan_vdot(ytn_plan_t *p, const Tensor &A, const Tensor &B, std::string &err) {
  if (A.nsym != B.nsym || std::memcmp(A.mod, B.mod, sizeof(A.mod)) != 0 || A.rank != B.rank) {
    err = "tensors of different symmetry or rank";
    return YTN_E_INVALID;
  }
  for (int i = 0; i < A.rank; i++)
    if (A.sig[i] != B.sig[i]) { err = "tensors with different leg signatures"; return YTN_E_SIGNATURE; }
  for (int i = 0; i < A.rank; i++) {
    auto da = leg_dims(A, i), db = leg_dims(B, i);
    for (auto &kv : da) {
      auto it = db.find(kv.first);
      if (it != db.end() && it->second != kv.second) {
        err = "leg " + std::to_string(i) + " charge " + keystr(kv.first) + ": dimension " +
              std::to_string(kv.second) + " vs " + std::to_string(it->second);
        return YTN_E_DIM_MISMATCH;
      }
    }
    const bool fa = (bool)A.fus[i], fb = (bool)B.fus[i];
    if (fa != fb || (fa && !fusion_equal(*A.fus[i], *B.fus[i]))) {
      err = "leg " + std::to_string(i) + ": fusion records differ";
      return YTN_E_FUSION_MISMATCH;
    }
  }
  if (A.dtype != B.dtype) { err = "scalar product of a real and a complex tensor"; return YTN_E_UNSUPPORTED; }
  // complex: runs of doubles (pairs), <A, B> = sum conj(a) b
  const int cw = A.dtype == YTN_COMPLEX128 ? 2 : 1;
  p->cw = cw;
  // common blocks: both block lists are in canonical (ascending) order
  const size_t w = (size_t)A.rank * A.nsym;
  auto key_of = [w](const Tensor &T, int64_t b) { return Key(T.t.begin() + b * w, T.t.begin() + (b + 1) * w); };
  p->vd_pieces.clear();
  p->vd_chunks.clear();
  int64_t common = 0;
  for (int64_t i = 0, j = 0; i < A.nblocks && j < B.nblocks;) {
    const Key ka = key_of(A, i), kb = key_of(B, j);
    if (ka < kb) { i++; continue; }
    if (kb < ka) { j++; continue; }
    const int64_t n = A.elems(i), nd = cw * n;
    for (int64_t e = 0; e < nd; e += kVdotPiece)
      p->vd_pieces.push_back({cw * A.off[i] + e, cw * B.off[j] + e, (int32_t)std::min<int64_t>(kVdotPiece, nd - e), 0});
    common += n;
    i++;
    j++;
  }
  // CTA shares: consecutive pieces, at most kVdotChunk elements and 64 pieces
  for (size_t k = 0; k < p->vd_pieces.size();) {
    size_t m = k;
    int64_t tot = 0;
    while (m < p->vd_pieces.size() && m - k < 64 && tot + p->vd_pieces[m].len <= kVdotChunk) tot += p->vd_pieces[m++].len;
    p->vd_chunks.push_back({(int32_t)k, (int32_t)(m - k)});
    k = m;
  }
  if (p->vd_chunks.size() > (size_t)INT32_MAX) { err = "scalar product too large"; return YTN_E_UNSUPPORTED; }
  // output: a rank-0 tensor with one element
  Tensor &C = p->out;
  C = Tensor();
  C.nsym = A.nsym;
  for (int c = 0; c < A.nsym; c++) C.mod[c] = A.mod[c];
  C.rank = 0;
  C.dtype = A.dtype;
  C.nblocks = 1;
  C.off.push_back(0);
  C.size = 1;
  p->flops = 2.0 * (double)common * (cw == 2 ? 4 : 1);
  p->moved = common;
  p->kind = Kind::Vdot;
  p->a_size = A.size;
  p->b_size = B.size;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Fermionic swap gate
// ---------------------------------------------------------------------------

// Sec. IV: at a crossing of two lines in the fermionic order, a swap gate
// changes the sign of the blocks whose charges are odd on both lines. A
// group's parity is the sum over its legs of the fermionic components of the
// leg's charge, modulo 2 (a signature does not change a parity). The output
// has a's structure and layout; each block is one copy, negated or not.
ytn_status plan_swap_gate(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                          uint32_t fermionic, std::string &err) {
  if (ngroups != 2) { err = "a swap gate takes two groups of legs"; return YTN_E_INVALID; }
  std::vector<int> seen(A.rank, 0);
  std::vector<int> g[2];
  int pos = 0;
  for (int k = 0; k < 2; k++) {
    if (group_size[k] < 1 || pos + group_size[k] > A.rank) { err = "bad group sizes"; return YTN_E_INVALID; }
    for (int i = 0; i < group_size[k]; i++) {
      const int l = order[pos++];
      if (l < 0 || l >= A.rank || seen[l]) { err = "swap-gate groups must be disjoint legs in range"; return YTN_E_INVALID; }
      seen[l] = 1;
      g[k].push_back(l);
    }
  }
  const uint32_t mask = fermionic == 0 ? ((1u << A.nsym) - 1u) : (fermionic & ~YTN_FERMIONIC_EXPLICIT);
  if (fermionic != 0 && !(fermionic & YTN_FERMIONIC_EXPLICIT)) {
    err = "an explicit fermionic set needs YTN_FERMIONIC_EXPLICIT";
    return YTN_E_INVALID;
  }
  if (mask >> A.nsym) { err = "fermionic flag of a component the symmetry does not have"; return YTN_E_INVALID; }
  for (int c = 0; c < A.nsym; c++)
    if (((mask >> c) & 1u) && (A.mod[c] % 2) != 0) {
      err = "a fermionic component must be U(1) or Z_m with m even";
      return YTN_E_INVALID;
    }
  auto parity = [&](int64_t b, const std::vector<int> &legs) {
    int64_t s = 0;
    for (int l : legs) {
      const int32_t *q = A.charge(b, l);
      for (int c = 0; c < A.nsym; c++)
        if ((mask >> c) & 1u) s += q[c];
    }
    return (int)(((s % 2) + 2) % 2);
  };
  p->out = A;
  p->cw = A.dtype == YTN_COMPLEX128 ? 2 : 1;
  p->jobs.clear();
  p->items.clear();
  p->moved = 0;
  for (int64_t b = 0; b < A.nblocks; b++) {
    const int64_t n = A.elems(b);
    const bool neg = parity(b, g[0]) == 1 && parity(b, g[1]) == 1;
    ytn_status s = add_copy(p, {{n, 1, 1}}, A.off[b], A.off[b], err, neg ? 1 : 0);
    if (s != YTN_OK) return s;
    p->moved += n;
  }
  p->items_a_begin = 0;
  make_items(p, 0, p->jobs.size());
  p->items_a_end = (int64_t)p->items.size();
  p->zero_out = false;
  p->flops = 0.0;
  p->kind = Kind::Swap;
  p->a_size = A.size;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Conjugation
// ---------------------------------------------------------------------------

// Sec. II.A footnote: conjugation flips every leg's signature (so n becomes -n,
// and each fusion record's constituent signatures flip) and complex-conjugates
// the elements. Blocks keep their charges and places; complex data is copied
// with its imaginary parts negated, real data is copied as it is.
ytn_status plan_conj(ytn_plan_t *p, const Tensor &A, std::string &err) {
  p->out = A;
  Tensor &C = p->out;
  for (int i = 0; i < C.rank; i++) {
    C.sig[i] = -A.sig[i];
    if (A.fus[i]) {
      auto F = std::make_shared<Fusion>(*A.fus[i]);
      for (int j = 0; j < F->nlegs; j++) F->sig[j] = -F->sig[j];
      C.fus[i] = F;
    }
  }
  for (int c = 0; c < C.nsym; c++) C.n[c] = reduce(-(int64_t)A.n[c], A.mod[c]);
  p->cw = A.dtype == YTN_COMPLEX128 ? 2 : 1;
  p->jobs.clear();
  p->items.clear();
  p->moved = 0;
  for (int64_t b = 0; b < A.nblocks; b++) {
    const int64_t n = A.elems(b);
    ytn_status s = add_copy(p, {{n, 1, 1}}, A.off[b], A.off[b], err, p->cw == 2 ? 2 : 0);
    if (s != YTN_OK) return s;
    p->moved += n;
  }
  p->items_a_begin = 0;
  make_items(p, 0, p->jobs.size());
  p->items_a_end = (int64_t)p->items.size();
  p->zero_out = false;
  p->flops = 0.0;
  p->kind = Kind::Conj;
  p->a_size = A.size;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Block-diagonal SVD and leg slicing
// ---------------------------------------------------------------------------

// Sec. III (CTM): the fused enlarged corner is block diagonal in the charge
// sectors and its SVD is one dense SVD per block. Rows are the combinations of
// the row legs' charges, grouped by their signed sum c (ascending, each row-major
// over its legs), columns likewise; M_c is gathered row-major into the workspace
// and factored by the dense solver. Outputs: U (row legs, new leg of signature -1),
// S (new leg +1, new leg -1; a k x k diagonal block per sector), V (new leg +1,
// col legs); the new leg has charge c and dimension k_c = min(m_c, n_c).
// eig: the Hermitian eigendecomposition instead (column legs dual to the row
// legs, n = 0, square sectors; M_c = U_c diag(w_c) U_c^H, w ascending): M_c is
// gathered column-major, the solver overwrites it with U_c, and there is no V.
static ytn_status plan_decomp(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                              bool eig, std::string &err);

ytn_status plan_svd(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                    std::string &err) {
  return plan_decomp(p, A, ngroups, group_size, order, false, err);
}

ytn_status plan_eigh(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                     std::string &err) {
  return plan_decomp(p, A, ngroups, group_size, order, true, err);
}

static ytn_status plan_decomp(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                              bool eig, std::string &err) {
  const int w = A.dtype == YTN_COMPLEX128 ? 2 : 1;   // doubles per element
  p->cw = w;   // the gathers and scatters below move whole (complex) elements
  if (ngroups != 2 || group_size[0] < 1 || group_size[1] < 1 || group_size[0] + group_size[1] != A.rank) {
    err = "an SVD takes two nonempty groups of legs: rows and columns";
    return YTN_E_INVALID;
  }
  std::vector<int> rowL(order, order + group_size[0]), colL(order + group_size[0], order + A.rank);
  {
    std::vector<int> seen(A.rank, 0);
    for (int l : rowL) if (l < 0 || l >= A.rank || seen[l]++) { err = "row/column legs must split the legs"; return YTN_E_INVALID; }
    for (int l : colL) if (l < 0 || l >= A.rank || seen[l]++) { err = "row/column legs must split the legs"; return YTN_E_INVALID; }
  }
  if ((int)rowL.size() + 1 > YTN_MAX_RANK || (int)colL.size() + 1 > YTN_MAX_RANK) {
    err = "SVD output rank too large";
    return YTN_E_UNSUPPORTED;
  }
  if (eig) {
    if (rowL.size() != colL.size()) { err = "eigh needs as many column legs as row legs"; return YTN_E_INVALID; }
    for (size_t i = 0; i < rowL.size(); i++)
      if (A.sig[rowL[i]] != -A.sig[colL[i]]) { err = "eigh needs column legs dual to the row legs"; return YTN_E_SIGNATURE; }
    for (int c = 0; c < A.nsym; c++)
      if (A.n[c] != 0) { err = "eigh needs total charge 0"; return YTN_E_CHARGE; }
  }
  const int nsym = A.nsym;
  struct Sec {
    std::map<Key, std::pair<int64_t, int64_t>> rows, cols;   // key -> (size, any block)
    std::vector<int64_t> blocks;
  };
  std::map<Key, Sec> secs;
  for (int64_t b = 0; b < A.nblocks; b++) {
    Key c(nsym, 0);
    for (int l : rowL)
      for (int q = 0; q < nsym; q++) c[q] = reduce((int64_t)c[q] + (int64_t)A.sig[l] * A.charge(b, l)[q], A.mod[q]);
    Sec &sc = secs[c];
    sc.rows.emplace(sub_charges(A, b, rowL), std::make_pair(sub_elems(A, b, rowL), b));
    sc.cols.emplace(sub_charges(A, b, colL), std::make_pair(sub_elems(A, b, colL), b));
    sc.blocks.push_back(b);
  }
  // output structures
  Tensor U, S, V;
  for (Tensor *T : {&U, &S, &V}) {
    T->nsym = nsym;
    std::memcpy(T->mod, A.mod, sizeof(T->mod));
  }
  U.rank = (int)rowL.size() + 1;
  for (size_t i = 0; i < rowL.size(); i++) {
    U.sig[i] = A.sig[rowL[i]];
    copy_fusion(A.fus[rowL[i]].get(), U.fus[i]);
  }
  U.sig[rowL.size()] = -1;
  U.dtype = V.dtype = A.dtype;   // S is real
  S.rank = 2;
  S.sig[0] = 1;
  S.sig[1] = -1;
  V.rank = (int)colL.size() + 1;
  V.sig[0] = 1;
  for (size_t i = 0; i < colL.size(); i++) {
    V.sig[i + 1] = A.sig[colL[i]];
    copy_fusion(A.fus[colL[i]].get(), V.fus[i + 1]);
  }
  std::memcpy(V.n, A.n, sizeof(V.n));
  std::vector<OutBlock> ub, sb, vb;
  struct Place { int64_t sec; int64_t off; int64_t blk; };
  std::vector<Place> uplace, vplace;   // per output block id: its sector, row/col offset, a source block
  p->svd_sec.clear();
  size_t off = 0;
  auto align32 = [](int64_t e) { return (e + 31) / 32 * 32; };
  std::vector<std::map<Key, int64_t>> roff(secs.size()), coff(secs.size());
  int64_t si = 0;
  int64_t covered = 0, need = 0;
  for (auto &kv : secs) {
    SvdSector sv{};
    for (auto &r : kv.second.rows) { roff[si][r.first] = sv.m; sv.m += r.second.first; }
    for (auto &c : kv.second.cols) { coff[si][c.first] = sv.n; sv.n += c.second.first; }
    if (eig) {
      // square, columns in the order of the rows (dual legs: the same tuples)
      bool same = kv.second.rows.size() == kv.second.cols.size();
      for (auto r = kv.second.rows.begin(), c = kv.second.cols.begin(); same && r != kv.second.rows.end(); ++r, ++c)
        same = r->first == c->first && r->second.first == c->second.first;
      if (!same) { err = "eigh: a sector whose columns do not match its rows"; return YTN_E_DIM_MISMATCH; }
    }
    sv.k = std::min(sv.m, sv.n);
    sv.trans = (eig || sv.n < sv.m) ? 1 : 0;
    if (sv.m > INT32_MAX || sv.n > INT32_MAX) { err = "sector too large"; return YTN_E_UNSUPPORTED; }
    sv.m_off = (int64_t)off;
    off += align32(sv.m * sv.n);
    need += sv.m * sv.n;
    p->svd_sec.push_back(sv);
    for (auto &r : kv.second.rows) {
      OutBlock ob;
      ob.key = r.first;
      ob.key.insert(ob.key.end(), kv.first.begin(), kv.first.end());
      for (int l : rowL) ob.D.push_back(A.dim(r.second.second, l));
      ob.D.push_back(sv.k);
      ob.id = (int64_t)uplace.size();
      ub.push_back(ob);
      uplace.push_back({si, roff[si][r.first], r.second.second});
    }
    {
      OutBlock ob;
      ob.key = kv.first;
      ob.key.insert(ob.key.end(), kv.first.begin(), kv.first.end());
      ob.D = {sv.k, sv.k};
      ob.id = (int64_t)sb.size();
      sb.push_back(ob);
    }
    for (auto &c : kv.second.cols) {
      if (eig) break;
      OutBlock ob;
      ob.key = kv.first;
      ob.key.insert(ob.key.end(), c.first.begin(), c.first.end());
      ob.D.push_back(sv.k);
      for (int l : colL) ob.D.push_back(A.dim(c.second.second, l));
      ob.id = (int64_t)vplace.size();
      vb.push_back(ob);
      vplace.push_back({si, coff[si][c.first], c.second.second});
    }
    si++;
  }
  p->svd_m_doubles = w * off;
  for (auto &sv : p->svd_sec) {
    if (eig) { sv.up_off = sv.vp_off = sv.m_off; continue; }   // U overwrites the matrix
    sv.up_off = (int64_t)off;
    off += align32(sv.n * sv.k);
  }
  for (auto &sv : p->svd_sec) {
    if (eig) continue;
    sv.vp_off = (int64_t)off;
    off += align32(sv.m * sv.k);
  }
  off *= w;   // from here on, doubles
  for (auto &sv : p->svd_sec) { sv.s_off = (int64_t)off; off += align32(sv.k); }
  p->svd_info_off = off;                       // one int per sector (as doubles: rounded up)
  off += align32(((int64_t)p->svd_sec.size() + 1) / 2 + 1);
  p->svd_ws_doubles = off;                     // the solver's buffer follows (size set by the device side)
  std::vector<int64_t> uo, so, vo;
  finalize_out(U, ub, uo);
  finalize_out(S, sb, so);
  finalize_out(V, vb, vo);
  p->jobs.clear();
  p->items.clear();
  p->moved = 0;
  // gather A -> M_c (row-major, ld = n; column-major, ld = m, when trans)
  si = 0;
  for (auto &kv : secs) {
    const SvdSector &sv = p->svd_sec[si];
    for (int64_t b : kv.second.blocks) {
      const auto st = block_strides(A, b);
      std::vector<Dim> dims;
      int64_t acc = 1;
      std::vector<int64_t> rs(rowL.size()), cs(colL.size());
      for (int i = (int)rowL.size() - 1; i >= 0; i--) { rs[i] = acc; acc *= A.dim(b, rowL[i]); }
      acc = 1;
      for (int i = (int)colL.size() - 1; i >= 0; i--) { cs[i] = acc; acc *= A.dim(b, colL[i]); }
      const int64_t rstep = sv.trans ? 1 : sv.n, cstep = sv.trans ? sv.m : 1;
      for (size_t i = 0; i < rowL.size(); i++) dims.push_back({A.dim(b, rowL[i]), st[rowL[i]], rs[i] * rstep});
      for (size_t i = 0; i < colL.size(); i++) dims.push_back({A.dim(b, colL[i]), st[colL[i]], cs[i] * cstep});
      const int64_t dst = sv.m_off + roff[si][sub_charges(A, b, rowL)] * rstep + coff[si][sub_charges(A, b, colL)] * cstep;
      ytn_status s = add_copy(p, dims, A.off[b], dst, err);
      if (s != YTN_OK) return s;
      covered += A.elems(b);
      p->moved += A.elems(b);
    }
    si++;
  }
  p->svd_zero_m = covered < need;
  const size_t j0 = 0, j1 = p->jobs.size();
  p->items_a_begin = 0;
  make_items(p, j0, j1);
  p->items_a_end = (int64_t)p->items.size();
  // U blocks from F_m (m x k, column-major): element (row r, j) at vp_off + j*m + r
  for (size_t id = 0; id < uplace.size(); id++) {
    const Place &pl = uplace[id];
    const SvdSector &sv = p->svd_sec[pl.sec];
    const int64_t rows = sub_elems(A, pl.blk, rowL);
    ytn_status s = add_copy(p, {{rows, 1, sv.k}, {sv.k, sv.m, 1}}, sv.vp_off + pl.off, uo[id], err);
    if (s != YTN_OK) return s;
  }
  const size_t j2 = p->jobs.size();
  p->items_b_begin = (int64_t)p->items.size();
  make_items(p, j1, j2);
  p->items_b_end = (int64_t)p->items.size();
  // V blocks from F_n (n x k, column-major): element (j, col c) at up_off + j*n + c
  for (size_t id = 0; id < vplace.size(); id++) {
    const Place &pl = vplace[id];
    const SvdSector &sv = p->svd_sec[pl.sec];
    const int64_t cols = sub_elems(A, pl.blk, colL);
    ytn_status s = add_copy(p, {{sv.k, sv.n, cols}, {cols, 1, 1}}, sv.up_off + pl.off, vo[id], err);
    if (s != YTN_OK) return s;
  }
  const size_t j3 = p->jobs.size();
  p->items_c_begin = (int64_t)p->items.size();
  make_items(p, j2, j3);
  p->items_c_end = (int64_t)p->items.size();
  // S diagonals from the singular-value vectors (real; the rest of S is zero)
  p->cw = 1;
  for (size_t id = 0; id < p->svd_sec.size(); id++) {
    const SvdSector &sv = p->svd_sec[id];
    if (sv.k == 0) continue;
    ytn_status s = add_copy(p, {{sv.k, 1, sv.k + 1}}, sv.s_off, so[id], err);
    if (s != YTN_OK) return s;
  }
  const size_t j4 = p->jobs.size();
  p->items_s_begin = (int64_t)p->items.size();
  make_items(p, j3, j4);
  p->items_s_end = (int64_t)p->items.size();
  // complex data: the solver factors X = M^T (or M) as U_x S V_x^H, so that
  // M = conj(V_x) S U_x^T (or U_x S conj(V_x)^T): the factor F_m (or F_n) is
  // conjugated in place before the scatters (imaginary parts negated)
  p->cw = w;
  if (w == 2 && !eig)
    for (const SvdSector &sv : p->svd_sec) {
      if (sv.k == 0) continue;
      const int64_t o = sv.trans ? sv.up_off : sv.vp_off, n = sv.trans ? sv.n * sv.k : sv.m * sv.k;
      ytn_status s = add_copy(p, {{n, 1, 1}}, o, o, err, 2);
      if (s != YTN_OK) return s;
    }
  p->items_h_begin = (int64_t)p->items.size();
  make_items(p, j4, p->jobs.size());
  p->items_h_end = (int64_t)p->items.size();
  p->out = U;
  if (eig) p->outs = {S};
  else p->outs = {S, V};
  p->kind = eig ? Kind::Eigh : Kind::Svd;
  p->a_size = A.size;
  double fl = 0.0;
  for (auto &sv : p->svd_sec) fl += 4.0 * (double)sv.m * sv.n * sv.k;   // nominal dense SVD work
  p->flops = fl;
  return YTN_OK;
}

// The first keep[c] indices of every sector c of the legs `axes` (other legs
// whole); blocks with a sector kept at 0 are dropped. Truncates U, S and V to the
// kept singular values.
ytn_status plan_slice(ytn_plan_t *p, const Tensor &A, int naxes, const int *axes, int64_t nkeep,
                      const int32_t *keep_t, const int64_t *keep_D, std::string &err) {
  if (naxes < 1 || naxes > A.rank) { err = "naxes out of range"; return YTN_E_INVALID; }
  if (nkeep < 0 || (nkeep > 0 && (!keep_t || !keep_D))) { err = "null keep table"; return YTN_E_INVALID; }
  std::vector<int> ax(axes, axes + naxes);
  for (int a : ax)
    if (a < 0 || a >= A.rank || std::count(ax.begin(), ax.end(), a) != 1) { err = "bad sliced legs"; return YTN_E_INVALID; }
  std::map<Key, int64_t> keep;
  for (int64_t i = 0; i < nkeep; i++) {
    if (keep_D[i] < 0) { err = "negative kept dimension"; return YTN_E_INVALID; }
    Key q(keep_t + i * A.nsym, keep_t + (i + 1) * A.nsym);
    for (int c = 0; c < A.nsym; c++) q[c] = reduce(q[c], A.mod[c]);
    keep[q] = keep_D[i];
  }
  Tensor &C = p->out;
  C = A;
  C.t.clear();
  C.D.clear();
  C.off.clear();
  C.bstr.clear();
  p->cw = A.dtype == YTN_COMPLEX128 ? 2 : 1;
  std::vector<OutBlock> ob;
  std::vector<int64_t> src;
  for (int64_t b = 0; b < A.nblocks; b++) {
    OutBlock o;
    o.key = Key(&A.t[(size_t)b * A.rank * A.nsym], &A.t[(size_t)(b + 1) * A.rank * A.nsym]);
    bool ok = true;
    for (int i = 0; i < A.rank; i++) {
      int64_t d = A.dim(b, i);
      if (std::find(ax.begin(), ax.end(), i) != ax.end()) {
        auto it = keep.find(Key(A.charge(b, i), A.charge(b, i) + A.nsym));
        d = std::min(d, it == keep.end() ? 0 : it->second);
      }
      if (d == 0) ok = false;
      o.D.push_back(d);
    }
    if (!ok) continue;
    o.id = (int64_t)src.size();
    src.push_back(b);
    ob.push_back(o);
  }
  std::vector<int64_t> off_of_id;
  std::vector<OutBlock> sorted = ob;
  finalize_out(C, sorted, off_of_id);
  p->jobs.clear();
  p->items.clear();
  p->moved = 0;
  for (size_t id = 0; id < ob.size(); id++) {
    const int64_t b = src[id];
    const auto st = block_strides(A, b);
    std::vector<Dim> dims;
    int64_t acc = 1;
    std::vector<int64_t> ds(A.rank);
    for (int i = A.rank - 1; i >= 0; i--) { ds[i] = acc; acc *= ob[id].D[i]; }
    for (int i = 0; i < A.rank; i++) dims.push_back({ob[id].D[i], st[i], ds[i]});
    ytn_status s = add_copy(p, dims, A.off[b], off_of_id[id], err);
    if (s != YTN_OK) return s;
    p->moved += acc;
  }
  p->items_a_begin = 0;
  make_items(p, 0, p->jobs.size());
  p->items_a_end = (int64_t)p->items.size();
  p->zero_out = false;
  p->flops = 0.0;
  p->kind = Kind::Slice;
  p->a_size = A.size;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Tensor structure from legs (the paper's rand)
// ---------------------------------------------------------------------------

// Every block (rho_1 .. rho_r) with sum_i s_i rho_i = n: the first r - 1 legs are
// enumerated, the last leg's charge follows from the rule and is looked up.
ytn_status plan_blocks(ytn_plan_t *p, const ytn_sym &sym, int rank, const ytn_leg *legs, const int32_t *n,
                       std::string &err) {
  if (sym.nsym < 1 || sym.nsym > YTN_MAX_SYM) { err = "nsym out of range"; return YTN_E_INVALID; }
  if (rank < 1 || rank > YTN_MAX_RANK || !legs || !n) { err = "rank out of range or null legs"; return YTN_E_INVALID; }
  const int nsym = sym.nsym;
  Tensor C;
  C.nsym = nsym;
  for (int c = 0; c < nsym; c++) {
    if (sym.mod[c] < 0 || sym.mod[c] == 1) { err = "modulus must be 0 (U(1)) or >= 2"; return YTN_E_INVALID; }
    C.mod[c] = sym.mod[c];
    C.n[c] = reduce(n[c], C.mod[c]);
  }
  C.rank = rank;
  std::vector<std::vector<Key>> ch(rank);
  std::vector<std::vector<int64_t>> dims(rank);
  for (int l = 0; l < rank; l++) {
    const ytn_leg &L = legs[l];
    if ((L.sig != 1 && L.sig != -1) || L.ncharges < 0 || (L.ncharges > 0 && (!L.t || !L.D))) {
      err = "bad leg " + std::to_string(l);
      return YTN_E_INVALID;
    }
    C.sig[l] = L.sig;
    for (int i = 0; i < L.ncharges; i++) {
      Key q(L.t + (size_t)i * nsym, L.t + (size_t)(i + 1) * nsym);
      for (int c = 0; c < nsym; c++) q[c] = reduce(q[c], C.mod[c]);
      if (L.D[i] < 1 || L.D[i] > ((int64_t)1 << 30)) { err = "leg dimension out of range"; return YTN_E_INVALID; }
      if (i > 0 && !(ch[l].back() < q)) { err = "leg charges must ascend and be distinct"; return YTN_E_INVALID; }
      ch[l].push_back(q);
      dims[l].push_back(L.D[i]);
    }
  }
  std::map<Key, int> last;
  for (size_t i = 0; i < ch[rank - 1].size(); i++) last[ch[rank - 1][i]] = (int)i;
  std::vector<OutBlock> ob;
  std::vector<int> idx(rank, 0);
  const int r1 = rank - 1;
  bool empty = false;
  for (int l = 0; l < r1; l++) empty = empty || ch[l].empty();
  while (!empty) {
    // the last leg's charge: s_last q = n - sum_{l < last} s_l q_l
    Key need(nsym, 0);
    for (int c = 0; c < nsym; c++) {
      int64_t acc = C.n[c];
      for (int l = 0; l < r1; l++) acc -= (int64_t)C.sig[l] * ch[l][idx[l]][c];
      need[c] = reduce(acc * C.sig[r1], C.mod[c]);
    }
    auto it = last.find(need);
    if (it != last.end()) {
      OutBlock o;
      o.id = (int64_t)ob.size();
      for (int l = 0; l < r1; l++) {
        o.key.insert(o.key.end(), ch[l][idx[l]].begin(), ch[l][idx[l]].end());
        o.D.push_back(dims[l][idx[l]]);
      }
      o.key.insert(o.key.end(), need.begin(), need.end());
      o.D.push_back(dims[r1][it->second]);
      ob.push_back(o);
      if (ob.size() > (size_t)INT32_MAX) { err = "too many blocks"; return YTN_E_UNSUPPORTED; }
    }
    int l = r1 - 1;
    for (; l >= 0; l--) {
      if (++idx[l] < (int)ch[l].size()) break;
      idx[l] = 0;
    }
    if (l < 0) break;
  }
  std::vector<int64_t> off;
  finalize_out(C, ob, off);
  p->out = C;
  p->kind = Kind::Blocks;
  p->a_size = 0;
  p->flops = 0.0;
  return YTN_OK;
}

// ---------------------------------------------------------------------------
// Cache key and output view
// ---------------------------------------------------------------------------

static void put(std::string &s, const void *p, size_t n) { s.append((const char *)p, n); }

static void key_struct(std::string &s, const ytn_struct *t) {
  if (!t) { s += "N"; return; }
  put(s, &t->sym, sizeof(t->sym));
  put(s, &t->rank, sizeof(t->rank));
  put(s, t->sig, sizeof(t->sig));
  put(s, t->n, sizeof(t->n));
  put(s, &t->nblocks, sizeof(t->nblocks));
  put(s, &t->size, sizeof(t->size));
  put(s, &t->dtype, sizeof(t->dtype));
  const int nsym = t->sym.nsym > 0 && t->sym.nsym <= YTN_MAX_SYM ? t->sym.nsym : 0;
  const int rank = t->rank > 0 && t->rank <= YTN_MAX_RANK ? t->rank : 0;
  if (t->t) put(s, t->t, (size_t)t->nblocks * rank * nsym * sizeof(int32_t));
  if (t->D) put(s, t->D, (size_t)t->nblocks * rank * sizeof(int64_t));
  s += t->off ? "O" : "P";
  if (t->off) put(s, t->off, (size_t)t->nblocks * sizeof(int64_t));
  for (int i = 0; i < rank; i++) {
    const ytn_fusion *f = t->fus[i];
    if (!f) { s += "-"; continue; }
    s += "F";
    put(s, &f->nlegs, sizeof(f->nlegs));
    put(s, f->sig, sizeof(f->sig));
    put(s, &f->nentries, sizeof(f->nentries));
    const int m = f->nlegs > 0 && f->nlegs <= YTN_MAX_RANK ? f->nlegs : 0;
    if (f->nu) put(s, f->nu, (size_t)f->nentries * nsym * sizeof(int32_t));
    if (f->t) put(s, f->t, (size_t)f->nentries * m * nsym * sizeof(int32_t));
    if (f->D) put(s, f->D, (size_t)f->nentries * m * sizeof(int64_t));
  }
}

std::string plan_key(const ytn_op *op) {
  std::string s;
  put(s, &op->kind, sizeof(op->kind));
  put(s, &op->naxes, sizeof(op->naxes));
  put(s, op->axa, sizeof(op->axa));
  put(s, op->axb, sizeof(op->axb));
  put(s, &op->ngroups, sizeof(op->ngroups));
  put(s, op->group_size, sizeof(op->group_size));
  put(s, op->order, sizeof(op->order));
  if (op->kind == YTN_OP_SWAP_GATE) put(s, &op->fermionic, sizeof(op->fermionic));
  if (op->kind == YTN_OP_SLICE) {
    put(s, &op->nkeep, sizeof(op->nkeep));
    const int nsym = op->a && op->a->sym.nsym > 0 && op->a->sym.nsym <= YTN_MAX_SYM ? op->a->sym.nsym : 0;
    if (op->nkeep > 0 && op->keep_t) put(s, op->keep_t, (size_t)op->nkeep * nsym * sizeof(int32_t));
    if (op->nkeep > 0 && op->keep_D) put(s, op->keep_D, (size_t)op->nkeep * sizeof(int64_t));
  }
  key_struct(s, op->a);
  key_struct(s, op->b);
  return s;
}

void finish_output_view(ytn_plan_t *p) {
  make_view(p->out, p->out_view, p->out_fus_view);
  p->outs_view.assign(p->outs.size(), ytn_struct{});
  p->outs_fus_view.assign(p->outs.size(), {});
  for (size_t i = 0; i < p->outs.size(); i++) make_view(p->outs[i], p->outs_view[i], p->outs_fus_view[i]);
}

void make_view(const Tensor &C, ytn_struct &v, std::vector<ytn_fusion> &fv) {
  std::memset(&v, 0, sizeof(v));
  v.dtype = C.dtype;
  v.sym.nsym = C.nsym;
  for (int c = 0; c < YTN_MAX_SYM; c++) v.sym.mod[c] = C.mod[c];
  v.rank = C.rank;
  for (int i = 0; i < C.rank; i++) v.sig[i] = (int8_t)C.sig[i];
  for (int c = 0; c < YTN_MAX_SYM; c++) v.n[c] = C.n[c];
  v.nblocks = C.nblocks;
  v.t = C.t.data();
  v.D = C.D.data();
  v.off = C.off.data();
  v.size = C.size;
  fv.assign(C.rank, ytn_fusion{});
  for (int i = 0; i < C.rank; i++) {
    if (!C.fus[i]) continue;
    ytn_fusion &f = fv[i];
    const Fusion &F = *C.fus[i];
    f.nlegs = F.nlegs;
    for (int j = 0; j < F.nlegs; j++) f.sig[j] = (int8_t)F.sig[j];
    f.nentries = F.nentries;
    f.nu = F.nu.data();
    f.t = F.t.data();
    f.D = F.D.data();
    v.fus[i] = &f;
  }
}

}  // namespace ytn
