// Networks of tensors in the ncon convention (Sec. II.B: general networks are
// contracted through pairwise tensordot by the einsum / ncon convenience
// functions; labelling of Pfeifer, Evenbly, Singh and Vidal, 2015).
//
// Planning turns the network into a fixed list of library calls, each with its
// own cached plan: traces (a label twice on one tensor), pairwise tensordots
// (smallest remaining label first, over every label the two tensors share),
// outer products of what is left, and a final permutation of the legs into the
// order -1, -2, ... (a fuse with one leg per group). Intermediates live in the
// caller's workspace; the last call writes the caller's output. Execution only
// enqueues those calls on one stream.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "ytn.h"
#include "ytn_internal.hpp"

namespace {

enum StepKind { kTensordot = 1, kTrace = 2, kPermute = 3 };

// Operand ids: 0..n-1 are the caller's tensors, n + k is intermediate slot k,
// -1 is the caller's output.
struct Step {
  StepKind kind;
  ytn_plan_t *plan;
  int in0, in1, out;
};

struct Item {
  int id;
  const ytn_struct *st;
  std::vector<int> labels;
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

struct ytn_ncon_s {
  ytn_ctx *ctx = nullptr;
  int n = 0;
  std::vector<Step> steps;
  std::vector<size_t> slot_off;   // byte offsets of the intermediates in the workspace
  size_t slots_bytes = 0;
  double flops = 0.0;
  const ytn_struct *out = nullptr;

  ~ytn_ncon_s() {
    for (Step &s : steps) ytn_plan_release(s.plan);
  }
};

static ytn_status plan_step(ytn_ncon_t *nc, ytn_op &op, StepKind kind, int in0, int in1, Item &res) {
  ytn_plan_t *p = nullptr;
  ytn_status st = ytn_plan(nc->ctx, &op, &p);
  if (st != YTN_OK) return st;
  ytn_plan_info info;
  ytn_plan_get_info(p, &info);
  nc->flops += info.useful_flops;
  const ytn_struct *o = ytn_plan_output(p);
  nc->slot_off.push_back(nc->slots_bytes);
  nc->slots_bytes += align256((size_t)o->size * sizeof(double) * (o->dtype == YTN_COMPLEX128 ? 2 : 1));
  const int out = nc->n + (int)nc->slot_off.size() - 1;
  nc->steps.push_back({kind, p, in0, in1, out});
  res.id = out;
  res.st = o;
  return YTN_OK;
}

static ytn_status invalid(const char *msg) { return ytn::fail(YTN_E_INVALID, msg); }

extern "C" ytn_status ytn_ncon_plan(ytn_ctx *ctx, int32_t ntensors, const ytn_struct *const *tensors,
                                    const int32_t *labels, ytn_ncon_t **out) {
  if (!ctx || !tensors || !out || ntensors < 1) return invalid("null argument or empty network");
  *out = nullptr;
  std::vector<Item> items;
  std::map<int, int> count;
  int pos = 0;
  for (int i = 0; i < ntensors; i++) {
    if (!tensors[i] || tensors[i]->rank < 0 || tensors[i]->rank > YTN_MAX_RANK) return invalid("bad tensor");
    Item it{i, tensors[i], {}};
    for (int k = 0; k < tensors[i]->rank; k++) {
      const int x = labels[pos++];
      if (x == 0) return invalid("label 0");
      it.labels.push_back(x);
      count[x]++;
    }
    items.push_back(std::move(it));
  }
  int nneg = 0;
  for (auto &kv : count) {
    if (kv.first > 0 && kv.second != 2) return invalid("a positive label must appear twice");
    if (kv.first < 0) {
      if (kv.second != 1) return invalid("a negative label must appear once");
      nneg++;
    }
  }
  for (int k = 1; k <= nneg; k++)
    if (!count.count(-k)) return invalid("negative labels must be -1, -2, ... without gaps");
  ytn_ncon_t *nc = new (std::nothrow) ytn_ncon_t;
  if (!nc) return ytn::fail(YTN_E_NOMEM, "host allocation failed");
  nc->ctx = ctx;
  nc->n = ntensors;
  auto fail = [&](ytn_status s) {
    delete nc;
    return s;
  };
  try {
    for (;;) {
      int x = 0;
      for (auto &it : items)
        for (int y : it.labels)
          if (y > 0 && (x == 0 || y < x)) x = y;
      if (x == 0) break;
      std::vector<size_t> where;
      for (size_t i = 0; i < items.size(); i++)
        if (std::find(items[i].labels.begin(), items[i].labels.end(), x) != items[i].labels.end()) where.push_back(i);
      ytn_op op;
      std::memset(&op, 0, sizeof(op));
      if (where.size() == 1) {
        // every label this tensor carries twice, in ascending order
        Item &it = items[where[0]];
        std::set<int> twice;
        for (int y : it.labels)
          if (y > 0 && std::count(it.labels.begin(), it.labels.end(), y) == 2) twice.insert(y);
        op.kind = YTN_OP_TRACE;
        op.a = it.st;
        op.naxes = (int32_t)twice.size();
        std::vector<int> rest;
        int k = 0;
        for (int y : twice) {
          auto f = std::find(it.labels.begin(), it.labels.end(), y);
          auto l = std::find(f + 1, it.labels.end(), y);
          op.axa[k] = (int32_t)(f - it.labels.begin());
          op.axb[k] = (int32_t)(l - it.labels.begin());
          k++;
        }
        for (int y : it.labels)
          if (!twice.count(y)) rest.push_back(y);
        Item res{0, nullptr, rest};
        ytn_status st = plan_step(nc, op, kTrace, it.id, -1, res);
        if (st != YTN_OK) return fail(st);
        it = res;
        continue;
      }
      Item &A = items[where[0]];
      Item &B = items[where[1]];
      std::set<int> shared;
      for (int y : A.labels)
        if (y > 0 && std::find(B.labels.begin(), B.labels.end(), y) != B.labels.end()) shared.insert(y);
      op.kind = YTN_OP_TENSORDOT;
      op.a = A.st;
      op.b = B.st;
      op.naxes = (int32_t)shared.size();
      int k = 0;
      for (int y : shared) {
        op.axa[k] = (int32_t)(std::find(A.labels.begin(), A.labels.end(), y) - A.labels.begin());
        op.axb[k] = (int32_t)(std::find(B.labels.begin(), B.labels.end(), y) - B.labels.begin());
        k++;
      }
      std::vector<int> lc;
      for (int y : A.labels)
        if (!shared.count(y)) lc.push_back(y);
      for (int y : B.labels)
        if (!shared.count(y)) lc.push_back(y);
      Item res{0, nullptr, lc};
      ytn_status st = plan_step(nc, op, kTensordot, A.id, B.id, res);
      if (st != YTN_OK) return fail(st);
      items[where[0]] = res;
      items.erase(items.begin() + (std::ptrdiff_t)where[1]);
    }
    // outer products of the pieces left, in list order
    while (items.size() > 1) {
      ytn_op op;
      std::memset(&op, 0, sizeof(op));
      op.kind = YTN_OP_TENSORDOT;
      op.a = items[0].st;
      op.b = items[1].st;
      std::vector<int> lc = items[0].labels;
      lc.insert(lc.end(), items[1].labels.begin(), items[1].labels.end());
      Item res{0, nullptr, lc};
      ytn_status st = plan_step(nc, op, kTensordot, items[0].id, items[1].id, res);
      if (st != YTN_OK) return fail(st);
      items[0] = res;
      items.erase(items.begin() + 1);
    }
    Item &last = items[0];
    const int r = (int)last.labels.size();
    bool identity = true;
    for (int k = 0; k < r; k++) identity = identity && last.labels[k] == -(k + 1);
    if (identity && !nc->steps.empty()) {
      // the last call writes the caller's output; its slot is not needed
      nc->steps.back().out = -1;
      nc->slots_bytes = nc->slot_off.back();
      nc->slot_off.pop_back();
      nc->out = last.st;
    } else {
      if (r == 0) return fail(ytn::fail(YTN_E_UNSUPPORTED, "a network of one rank-0 tensor"));
      ytn_op op;
      std::memset(&op, 0, sizeof(op));
      op.kind = YTN_OP_FUSE;
      op.a = last.st;
      op.ngroups = r;
      for (int k = 0; k < r; k++) {
        op.group_size[k] = 1;
        op.order[k] = (int32_t)(std::find(last.labels.begin(), last.labels.end(), -(k + 1)) - last.labels.begin());
      }
      Item res{0, nullptr, {}};
      ytn_status st = plan_step(nc, op, kPermute, last.id, -1, res);
      if (st != YTN_OK) return fail(st);
      nc->steps.back().out = -1;
      nc->slots_bytes = nc->slot_off.back();
      nc->slot_off.pop_back();
      nc->out = res.st;
    }
  } catch (const std::bad_alloc &) {
    return fail(ytn::fail(YTN_E_NOMEM, "host allocation failed"));
  }
  *out = nc;
  return YTN_OK;
}

// einsum subscripts -> ncon labels: a letter on two legs is summed (numbered 1, 2,
// ... by first appearance), a letter on one leg is an output leg (-1, -2, ... in
// the order after "->", or alphabetical without it).
extern "C" ytn_status ytn_einsum_plan(ytn_ctx *ctx, const char *subscripts, int32_t ntensors,
                                      const ytn_struct *const *tensors, ytn_ncon_t **out) {
  if (!subscripts || !tensors || ntensors < 1) return invalid("null argument or empty network");
  std::string s;
  for (const char *c = subscripts; *c; c++)
    if (*c != ' ') s += *c;
  const size_t arrow = s.find("->");
  const std::string lhs = s.substr(0, arrow);
  std::vector<std::string> ins(1);
  for (char c : lhs) {
    if (c == ',') ins.emplace_back();
    else if ((c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z')) ins.back() += c;
    else return invalid("einsum subscripts: letters, commas and one arrow only");
  }
  if ((int)ins.size() != ntensors) return invalid("einsum subscripts: one letter group per tensor");
  std::map<char, int> count;
  for (auto &g : ins)
    for (char c : g) count[c]++;
  std::string outl;
  if (arrow != std::string::npos) {
    outl = s.substr(arrow + 2);
  } else {
    for (auto &kv : count)
      if (kv.second == 1) outl += kv.first;
  }
  std::set<char> once, seen;
  for (auto &kv : count) {
    if (kv.second > 2) return invalid("einsum subscripts: a letter on more than two legs");
    if (kv.second == 1) once.insert(kv.first);
  }
  for (char c : outl)
    if (!once.count(c) || !seen.insert(c).second) return invalid("einsum output must list every once-used letter once");
  if (seen.size() != once.size()) return invalid("einsum output must list every once-used letter once");
  std::map<char, int> lab;
  for (size_t k = 0; k < outl.size(); k++) lab[outl[k]] = -(int)(k + 1);
  int next = 1;
  std::vector<int32_t> labels;
  for (int i = 0; i < ntensors; i++) {
    if (!tensors[i] || tensors[i]->rank != (int)ins[i].size()) return invalid("einsum subscripts: one letter per leg");
    for (char c : ins[i]) {
      if (!lab.count(c)) lab[c] = next++;
      labels.push_back(lab[c]);
    }
  }
  return ytn_ncon_plan(ctx, ntensors, tensors, labels.data(), out);
}

extern "C" const ytn_struct *ytn_ncon_output(const ytn_ncon_t *nc) { return nc ? nc->out : nullptr; }

extern "C" ytn_status ytn_ncon_info(const ytn_ncon_t *nc, double *useful_flops, int32_t *ncalls) {
  if (!nc) return ytn::fail(YTN_E_INVALID, "null argument");
  if (useful_flops) *useful_flops = nc->flops;
  if (ncalls) *ncalls = (int32_t)nc->steps.size();
  return YTN_OK;
}

// Intermediates first, then one contraction workspace shared by the steps (they
// run one after another on the caller's stream).
static ytn_status gemm_bytes(const ytn_ncon_t *nc, ytn_precision prec, double rtol, size_t &bytes) {
  bytes = 0;
  for (const Step &s : nc->steps) {
    if (s.kind != kTensordot) continue;
    size_t b = 0;
    ytn_status st = ytn_workspace_size(s.plan, prec, rtol, &b);
    if (st != YTN_OK) return st;
    bytes = std::max(bytes, b);
  }
  return YTN_OK;
}

extern "C" ytn_status ytn_ncon_workspace_size(const ytn_ncon_t *nc, ytn_precision prec, double rtol, size_t *bytes) {
  if (!nc || !bytes) return ytn::fail(YTN_E_INVALID, "null argument");
  size_t g = 0;
  ytn_status st = gemm_bytes(nc, prec, rtol, g);
  if (st != YTN_OK) return st;
  *bytes = nc->slots_bytes + g;
  return YTN_OK;
}

extern "C" ytn_status ytn_ncon(ytn_ncon_t *nc, const double *const *data, double *out, ytn_precision prec, double rtol,
                               void *workspace, size_t workspace_bytes, ytn_stream stream) {
  if (!nc || !data || !out) return ytn::fail(YTN_E_INVALID, "null argument");
  size_t g = 0;
  ytn_status st = gemm_bytes(nc, prec, rtol, g);
  if (st != YTN_OK) return st;
  const size_t need = nc->slots_bytes + g;
  if (need && (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)))
    return ytn::fail(YTN_E_WORKSPACE, "workspace missing, too small or not 256-byte aligned");
  char *ws = static_cast<char *>(workspace);
  auto ptr = [&](int id) -> double * {
    if (id < 0) return out;
    if (id < nc->n) return const_cast<double *>(data[id]);
    return reinterpret_cast<double *>(ws + nc->slot_off[(size_t)(id - nc->n)]);
  };
  void *gws = g ? ws + nc->slots_bytes : nullptr;
  for (const Step &s : nc->steps) {
    switch (s.kind) {
      case kTensordot:
        st = ytn_tensordot(s.plan, ptr(s.in0), ptr(s.in1), ptr(s.out), prec, rtol, gws, g, nullptr, stream);
        break;
      case kTrace:
        st = ytn_trace(s.plan, ptr(s.in0), ptr(s.out), stream);
        break;
      case kPermute:
        st = ytn_fuse(s.plan, ptr(s.in0), ptr(s.out), stream);
        break;
    }
    if (st != YTN_OK) return st;
  }
  return YTN_OK;
}

extern "C" void ytn_ncon_release(ytn_ncon_t *nc) { delete nc; }
