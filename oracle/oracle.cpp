// Plain CPU oracle for the semiring Datalog fixpoint -- TEST INFRASTRUCTURE ONLY.
//
// Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
// file.  It shares no code with the CUDA engine: it has its own parser, its own
// relations (std::map of tuples), and its own semiring arithmetic in FP64.
//
// What it computes (Lobster, Sec. 3.1 "Provenance Semirings", Fig. 3 and the
// semiring table; Algorithm 1 for the iteration-until-no-growth loop):
//
//   F_0     = the loaded facts, duplicate rows merged with (+)  [(+) = oplus]
//   F_{k+1} = F_k updated with, for every head key h,
//               T(h) = (+) over all groundings g of a rule with head h,
//                      evaluated over F_k, of (x) of the tags of g's body facts
//   stop when an iteration changes nothing.
//
// The rules are split into strata (see stratify below), and the strata run one
// after another, each iterated to its fixpoint over the database the earlier
// strata left (Algorithm 1's loop over the strata of a RAM program).
//
// This is naive (not semi-naive) evaluation: every grounding over the whole
// database is enumerated in every iteration, which is the textbook definition
// of the least fixpoint.  How T(h) enters F_{k+1} depends on the semiring:
//
//   * unit, max-min-prob, diff-max-min (idempotent (+)):  F_{k+1}(h) = F_k(h) (+) T(h)
//     for every h (a missing key counts as 0).  This is the least fixpoint.
//   * add-mult-prob, diff-add-mult (non-idempotent (+)):  only keys absent from
//     F_k are added, with tag T(h); tags of existing keys never change.  This is
//     what semi-naive evaluation with size-based termination (Algorithm 1)
//     computes, and it terminates on cyclic graphs.
//
// Semirings (semiring table of Sec. 3.1 plus the probabilistic ones of Sec. 3.4):
//   0 unit           T = {true}, every tag is 1
//   1 max-min-prob   (+) = max, (x) = min on [0,1]
//   2 add-mult-prob  (+) = min(1, a + b), (x) = a * b on [0,1]
//   3 diff-max-min   tags (v, id); (+) keeps the larger (v, then smaller id),
//                    (x) keeps the smaller; d v / d p_id = 1
//   4 diff-add-mult  add-mult-prob carried with a forward-mode sparse gradient
//                    (dual number): d(a+b) = da + db, zero when a + b > 1;
//                    d(a*b) = a db + b da
//   5 top-1-proofs   (Sec. 5.3 "Limitations"; Sec. 3.4) a tag is one proof: the
//                    set of input facts of one derivation, at most `cap` of them
//                    (300 by default, the paper's limit); its probability is the
//                    product of its facts' probabilities.  (x) = union of the two
//                    proofs (a fact used twice counts once); (+) keeps the more
//                    likely proof.  Facts loaded without a probability have the
//                    empty proof (probability 1).  A union longer than the cap
//                    is an error.
//   6 diff-top-1-proofs  top-1-proofs with d P / d p_i = product of the
//                    proof's other facts' probabilities, for each fact i in it
//
// top-1-proofs details.  The probability of a proof is the product, in FP64,
// of its facts' probabilities in ascending input-fact id order, rounded once to
// f32 (the precision of every tag); (+) compares these f32 values.  When two
// different proofs of one key are equally likely the oracle keeps the one whose
// sorted id list is lexicographically smaller and counts the tie (orc_ties):
// the engine may keep either, so parity is checked on instances without ties.
//
// Rules may compute (Sec. 5.2): head arguments are u32 expressions over the
// body's variables (+, -, * modulo 2^32; unsigned /), and filters compare two
// such expressions with ==, !=, <, <=, >, >= (unsigned); see Expr below.
//
// Batched inputs (Sec. 4.3): facts carry a sample id and samples never join; the
// oracle states that directly by running the fixpoint once per sample (the
// samples on separate threads, their results gathered in sample order).
//
// ORACLE_MUTANT (default 0, the oracle itself): a positive value compiles one
// deliberate, plausible mistake into a separate library, so that
// tests/test_oracle_mutants.py can show that the pins of tests/test_oracle_pins.py
// catch it.  The mutants (a wrong operator, a dropped term, a transposed operand,
// a missing clamp, a wrong tie-break or policy, a skipped check, early stopping,
// samples that join) are listed at each #if below.
#include <algorithm>
#include <array>
#include <cctype>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

namespace {

constexpr int kMaxArity = 8;
constexpr uint32_t kNoId = 0xFFFFFFFFu;
using Tuple = std::array<uint32_t, kMaxArity>;
using Dual = std::map<uint32_t, double>;  // input-fact id -> partial derivative

enum Semiring { UNIT = 0, MAX_MIN = 1, ADD_MULT = 2, DIFF_MAX_MIN = 3, DIFF_ADD_MULT = 4, TOP1 = 5, DIFF_TOP1 = 6 };
bool is_top1(int sr) { return sr == TOP1 || sr == DIFF_TOP1; }

struct Tag {
  double v = 1.0;
  uint32_t id = kNoId;  // diff-max-min: the input fact that bounds v
  Dual d;               // diff-add-mult: d v / d p
  std::vector<uint32_t> proof;  // top-1-proofs: ascending input-fact ids
};

std::string g_err;
// top-1-proofs state of the current run: the probabilities are set before any
// sample runs and only read afterwards; the overflow flag and the tie count
// belong to the thread running a sample
std::vector<double> g_prob;  // input-fact id -> probability
uint32_t g_proof_cap = 300;
thread_local bool g_proof_overflow = false;
thread_local uint64_t g_ties = 0;

// probability of a proof: FP64 product in ascending id order, rounded to f32
double proof_prob(const std::vector<uint32_t>& proof) {
  double p = 1.0;
  for (uint32_t id : proof) p *= g_prob[id];
  return (double)(float)p;
}

// ---------------------------------------------------------------------------
// program text
// ---------------------------------------------------------------------------
struct Term {
  bool is_var = false;
  uint32_t value = 0;  // variable index or constant
};
struct Atom {
  std::string rel;
  std::vector<Term> args;
};
// Arithmetic over u32 values in head arguments and filters (Sec. 5.2: a
// projection or selection may compute): a leaf term, or a binary operation
// '+', '-', '*' (all modulo 2^32) or '/' (unsigned; a zero divisor drops the
// grounding).  A computed head value of 2^32 - 1 also drops the grounding (the
// engine reserves that value).
struct Expr {
  char op = 0;  // 0: leaf
  Term leaf;
  std::vector<Expr> kid;  // op != 0: the two operands
};
enum Cmp { CMP_EQ, CMP_NE, CMP_LT, CMP_LE, CMP_GT, CMP_GE };
struct Filter {
  Expr a, b;
  int cmp = CMP_EQ;
};
struct Rule {
  Atom head;
  std::vector<Expr> head_expr;  // per head argument (a leaf for a plain term)
  std::vector<Atom> body;
  std::vector<Filter> filters;
  int nvars = 0;
};

bool eval_expr(const Expr& e, const std::vector<uint32_t>& val, uint32_t& out) {
  if (!e.op) {
    out = e.leaf.is_var ? val[e.leaf.value] : e.leaf.value;
    return true;
  }
  uint32_t x, y;
  if (!eval_expr(e.kid[0], val, x) || !eval_expr(e.kid[1], val, y)) return false;
  switch (e.op) {
    case '+': out = x + y; break;
#if ORACLE_MUTANT == 16  // mutant: subtraction with its operands swapped
    case '-': out = y - x; break;
#else
    case '-': out = x - y; break;
#endif
    case '*': out = x * y; break;
    default:
      if (y == 0) return false;
      out = x / y;
  }
  return true;
}

bool compare_u32(int cmp, uint32_t x, uint32_t y) {
  switch (cmp) {
    case CMP_EQ: return x == y;
    case CMP_NE: return x != y;
#if ORACLE_MUTANT == 15  // mutant: '<' admits equality
    case CMP_LT: return x <= y;
#else
    case CMP_LT: return x < y;
#endif
    case CMP_LE: return x <= y;
    case CMP_GT: return x > y;
    default: return x >= y;
  }
}

struct Parser {
  const char* s;
  size_t i = 0;
  std::map<std::string, int> vars;
  explicit Parser(const char* text) : s(text) {}

  void skip() {
    for (;;) {
      while (s[i] && std::isspace((unsigned char)s[i])) i++;
      if (s[i] == '/' && s[i + 1] == '/') {
        while (s[i] && s[i] != '\n') i++;
      } else if (s[i] == '#') {
        while (s[i] && s[i] != '\n') i++;
      } else {
        return;
      }
    }
  }
  bool eat(const char* tok) {
    skip();
    size_t n = std::strlen(tok);
    if (std::strncmp(s + i, tok, n) == 0) {
      i += n;
      return true;
    }
    return false;
  }
  bool ident(std::string& out) {
    skip();
    if (!(std::isalpha((unsigned char)s[i]) || s[i] == '_')) return false;
    size_t j = i;
    while (std::isalnum((unsigned char)s[j]) || s[j] == '_') j++;
    out.assign(s + i, j - i);
    i = j;
    return true;
  }
  bool term(Term& t) {
    skip();
    if (std::isdigit((unsigned char)s[i])) {
      uint64_t v = 0;
      while (std::isdigit((unsigned char)s[i])) {
        v = v * 10 + (s[i] - '0');
        if (v > 0xFFFFFFFEull) return false;
        i++;
      }
      t.is_var = false;
      t.value = (uint32_t)v;
      return true;
    }
    std::string name;
    if (!ident(name)) return false;
    auto it = vars.find(name);
    int idx = it == vars.end() ? (int)vars.size() : it->second;
    if (it == vars.end()) vars[name] = idx;
    t.is_var = true;
    t.value = (uint32_t)idx;
    return true;
  }
  bool atom_after_name(const std::string& name, Atom& a) {
    a.rel = name;
    if (!eat("(")) return false;
    do {
      Term t;
      if (!term(t)) return false;
      a.args.push_back(t);
    } while (eat(","));
    return eat(")") && a.args.size() <= (size_t)kMaxArity;
  }
  // expr := product (('+' | '-') product)*; product := primary (('*' | '/') primary)*
  bool primary(Expr& e) {
    if (eat("(")) return expr(e) && eat(")");
    e.op = 0;
    return term(e.leaf);
  }
  bool product(Expr& e) {
    if (!primary(e)) return false;
    for (;;) {
      skip();
      const char c = s[i];
      if (c != '*' && c != '/') return true;
      i++;
      Expr n;
      n.op = c;
      n.kid.resize(2);
      n.kid[0] = e;
      if (!primary(n.kid[1])) return false;
      e = n;
    }
  }
  bool expr(Expr& e) {
    if (!product(e)) return false;
    for (;;) {
      skip();
      const char c = s[i];
      if (c != '+' && c != '-') return true;
      i++;
      Expr n;
      n.op = c;
      n.kid.resize(2);
      n.kid[0] = e;
      if (!product(n.kid[1])) return false;
      e = n;
    }
  }
  bool head(Rule& r) {
    std::string name;
    if (!ident(name)) return false;
    r.head.rel = name;
    if (!eat("(")) return false;
    do {
      Expr e;
      if (!expr(e)) return false;
      r.head.args.push_back(e.op ? Term{} : e.leaf);
      r.head_expr.push_back(e);
    } while (eat(","));
    return eat(")") && r.head.args.size() <= (size_t)kMaxArity;
  }
  bool rule(Rule& r) {
    vars.clear();
    if (!head(r)) return false;
    if (!eat(":-")) return false;
    do {
      skip();
      size_t save = i;
      std::string nm;
      if (ident(nm) && (skip(), s[i] == '(')) {
        Atom a;
        if (!atom_after_name(nm, a)) return false;
        r.body.push_back(a);
      } else {
        i = save;
        Filter f;
        if (!expr(f.a)) return false;
        if (eat("!=")) f.cmp = CMP_NE;
        else if (eat("==")) f.cmp = CMP_EQ;
        else if (eat("<=")) f.cmp = CMP_LE;
        else if (eat(">=")) f.cmp = CMP_GE;
        else if (eat("<")) f.cmp = CMP_LT;
        else if (eat(">")) f.cmp = CMP_GT;
        else return false;
        if (!expr(f.b)) return false;
        r.filters.push_back(f);
      }
    } while (eat(","));
    if (!eat(".")) return false;
    r.nvars = (int)vars.size();
    return !r.body.empty();
  }
  bool program(std::vector<Rule>& rules) {
    for (;;) {
      skip();
      if (!s[i]) return true;
      Rule r;
      if (!rule(r)) return false;
      rules.push_back(r);
    }
  }
};

// ---------------------------------------------------------------------------
// semiring arithmetic on tags (FP64)
// ---------------------------------------------------------------------------
// a "greater than" b in the diff-max-min order: larger value, then smaller id.
bool dmm_greater(const Tag& a, const Tag& b) {
  if (a.v != b.v) return a.v > b.v;
#if ORACLE_MUTANT == 3  // mutant: ties go to the larger input-fact id
  return a.id > b.id;
#endif
  return a.id < b.id;
}

Tag otimes(int sr, const Tag& a, const Tag& b) {
  Tag r;
  switch (sr) {
    case UNIT: r.v = 1.0; break;
#if ORACLE_MUTANT == 1  // mutant: max-min (x) takes the larger tag
    case MAX_MIN: r.v = std::max(a.v, b.v); break;
#else
    case MAX_MIN: r.v = std::min(a.v, b.v); break;
#endif
    case ADD_MULT: r.v = a.v * b.v; break;
#if ORACLE_MUTANT == 12  // mutant: diff-max-min (x) keeps the greater operand
    case DIFF_MAX_MIN: r = dmm_greater(a, b) ? a : b; break;
#else
    case DIFF_MAX_MIN: r = dmm_greater(a, b) ? b : a; break;
#endif
    case DIFF_ADD_MULT:
      r.v = a.v * b.v;
      for (auto& kv : a.d) r.d[kv.first] += b.v * kv.second;
#if ORACLE_MUTANT != 4  // mutant 4: the product rule's second term is dropped
      for (auto& kv : b.d) r.d[kv.first] += a.v * kv.second;
#endif
      break;
    case TOP1:
    case DIFF_TOP1:
#if ORACLE_MUTANT == 13  // mutant: the union keeps a fact used by both proofs twice
      std::merge(a.proof.begin(), a.proof.end(), b.proof.begin(), b.proof.end(), std::back_inserter(r.proof));
#else
      std::set_union(a.proof.begin(), a.proof.end(), b.proof.begin(), b.proof.end(), std::back_inserter(r.proof));
#endif
      if (r.proof.size() > g_proof_cap) {
        g_proof_overflow = true;
        r.proof.resize(g_proof_cap);
      }
      r.v = proof_prob(r.proof);
      break;
  }
  return r;
}

// top-1-proofs (+): the more likely proof; equally likely different proofs are
// a tie, resolved to the lexicographically smaller id list
bool top1_greater(const Tag& a, const Tag& b) {
#if ORACLE_MUTANT == 14  // mutant: (+) keeps the less likely proof
  if (a.v != b.v) return a.v < b.v;
#else
  if (a.v != b.v) return a.v > b.v;
#endif
  if (a.proof == b.proof) return false;
  g_ties++;
  return a.proof < b.proof;
}

// Accumulator for the (+) over the groundings of one head key.  For the
// add-mult semirings the clamp is applied once to the plain sum; this equals
// folding min(1, a + b) pairwise because all tags are non-negative.
struct Acc {
  bool any = false;
  Tag t;
  double sum = 0.0;
  Dual dsum;
};

void acc_add(int sr, Acc& acc, const Tag& g) {
  if (sr == ADD_MULT || sr == DIFF_ADD_MULT) {
    acc.sum += g.v;
    if (sr == DIFF_ADD_MULT)
      for (auto& kv : g.d) acc.dsum[kv.first] += kv.second;
    acc.any = true;
    return;
  }
  if (!acc.any) {
    acc.t = g;
    acc.any = true;
    return;
  }
  switch (sr) {
    case UNIT: break;
    case MAX_MIN: acc.t.v = std::max(acc.t.v, g.v); break;
    case DIFF_MAX_MIN:
      if (dmm_greater(g, acc.t)) acc.t = g;
      break;
    case TOP1:
    case DIFF_TOP1:
      if (top1_greater(g, acc.t)) acc.t = g;
      break;
  }
}

Tag acc_value(int sr, const Acc& acc) {
  if (sr == ADD_MULT || sr == DIFF_ADD_MULT) {
    Tag r;
#if ORACLE_MUTANT == 2  // mutant: (+) without the clamp to 1
    r.v = acc.sum;
#else
    r.v = std::min(1.0, acc.sum);
#endif
#if ORACLE_MUTANT == 5  // mutant: the derivative survives a clamped (+)
    if (sr == DIFF_ADD_MULT) r.d = acc.dsum;
#else
    if (sr == DIFF_ADD_MULT && !(acc.sum > 1.0)) r.d = acc.dsum;  // clamped: derivative 0
#endif
    return r;
  }
  return acc.t;
}

bool tag_equal(int sr, const Tag& a, const Tag& b) {
  if (sr == DIFF_MAX_MIN) return a.v == b.v && a.id == b.id;
  if (is_top1(sr)) return a.v == b.v && a.proof == b.proof;
  return a.v == b.v;
}

// ---------------------------------------------------------------------------
// strata (Sec. 3.1: a RAM program is a sequence of strata, run one after
// another, each to its own fixpoint; Algorithm 1's outer loop)
// ---------------------------------------------------------------------------
// The paper's front-end hands the engine its strata without saying how they
// are formed.  Reading: the textbook stratification of a positive program.  A
// relation that heads some rule is derived; a derived relation h depends on
// every derived relation in the body of a rule with head h.  The strata are the
// strongly connected components of that graph -- relations that depend on each
// other, directly or through others, share one -- ordered so that a component
// comes after every component it depends on; each rule goes to its head's.
// Among components that are ready at the same point, the one whose first rule
// comes first in the program goes first.
std::vector<std::vector<size_t>> stratify(const std::vector<Rule>& rules) {
  std::vector<std::string> derived;  // in order of first appearance as a head
  for (const Rule& r : rules)
    if (std::find(derived.begin(), derived.end(), r.head.rel) == derived.end()) derived.push_back(r.head.rel);
  const size_t n = derived.size();
  auto id = [&](const std::string& name) -> int {
    for (size_t i = 0; i < n; i++)
      if (derived[i] == name) return (int)i;
    return -1;
  };
  // reach[a][b]: a depends on b through one or more rules
  std::vector<std::vector<char>> reach(n, std::vector<char>(n, 0));
  for (const Rule& r : rules)
    for (const Atom& a : r.body) {
      const int b = id(a.rel);
      if (b >= 0) reach[id(r.head.rel)][b] = 1;
    }
  for (size_t m = 0; m < n; m++)  // transitive closure (Warshall)
    for (size_t a = 0; a < n; a++)
      if (reach[a][m])
        for (size_t b = 0; b < n; b++)
          if (reach[m][b]) reach[a][b] = 1;
  // component of a relation: itself and every relation it is mutually reachable with
  std::vector<int> comp(n, -1);
  int ncomp = 0;
  for (size_t a = 0; a < n; a++) {
    if (comp[a] >= 0) continue;
    comp[a] = ncomp;
    for (size_t b = a + 1; b < n; b++)
#if ORACLE_MUTANT == 18  // mutant: mutually recursive relations get separate strata
      if (false && reach[a][b] && reach[b][a]) comp[b] = ncomp;
#else
      if (reach[a][b] && reach[b][a]) comp[b] = ncomp;
#endif
    ncomp++;
  }
  // order: a component is placed once every component it depends on is placed
  std::vector<int> order;
  std::vector<char> placed(ncomp, 0);
  while ((int)order.size() < ncomp) {
    const size_t before = order.size();
    for (int c = 0; c < ncomp; c++) {
      if (placed[c]) continue;
      bool ready = true;
      for (size_t a = 0; a < n && ready; a++)
        if (comp[a] == c)
          for (size_t b = 0; b < n; b++)
            if (reach[a][b] && comp[b] != c && !placed[comp[b]]) ready = false;
      if (!ready) continue;
      placed[c] = 1;
      order.push_back(c);
      break;  // rescan from the first component, so ties go to program order
    }
    if (order.size() == before)  // no component ready: a dependency cycle across components
      for (int c = 0; c < ncomp; c++)  // (impossible unless mutant 18 split a component)
        if (!placed[c]) {
          placed[c] = 1;
          order.push_back(c);
          break;
        }
  }
#if ORACLE_MUTANT == 17  // mutant: strata run in reverse dependency order
  std::reverse(order.begin(), order.end());
#endif
  std::vector<std::vector<size_t>> strata;
  for (int c : order) {
    strata.emplace_back();
    for (size_t i = 0; i < rules.size(); i++)
      if (comp[id(rules[i].head.rel)] == c) strata.back().push_back(i);
  }
  return strata;
}

// ---------------------------------------------------------------------------
// naive fixpoint for one database (one sample)
// ---------------------------------------------------------------------------
using Relation = std::map<Tuple, Tag>;
using Database = std::map<std::string, Relation>;

struct Engine {
  int sr;
  const std::vector<Rule>& rules;
  Database db;
  int iterations = 0;

  Engine(int s, const std::vector<Rule>& r) : sr(s), rules(r) {}

  // Enumerate every grounding of rule `r` over `db` (body atoms in written
  // order, each matched against all facts of its relation consistent with the
  // variables bound so far).  Calls emit(head tuple, body fact tags).
  void groundings(const Rule& r, const std::function<void(const Tuple&, const std::vector<const Tag*>&)>& emit) {
    std::vector<uint32_t> val(r.nvars, 0);
    std::vector<char> bound(r.nvars, 0);
    std::vector<const Tag*> tags(r.body.size(), nullptr);
    // per atom: index from the values of columns bound on entry -> matching facts
    std::vector<std::vector<int>> bound_cols(r.body.size());
    {
      std::vector<char> b(r.nvars, 0);
      for (size_t j = 0; j < r.body.size(); j++) {
        const Atom& a = r.body[j];
        for (size_t c = 0; c < a.args.size(); c++)
          if (!a.args[c].is_var || b[a.args[c].value]) bound_cols[j].push_back((int)c);
        for (auto& t : a.args)
          if (t.is_var) b[t.value] = 1;
      }
    }
    using Key = std::vector<uint32_t>;
    std::vector<std::map<Key, std::vector<const std::pair<const Tuple, Tag>*>>> index(r.body.size());
    for (size_t j = 0; j < r.body.size(); j++) {
      auto it = db.find(r.body[j].rel);
      if (it == db.end()) return;
      for (auto& f : it->second) {
        Key k;
        for (int c : bound_cols[j]) k.push_back(f.first[c]);
        index[j][k].push_back(&f);
      }
    }
    std::function<void(size_t)> rec = [&](size_t j) {
      if (j == r.body.size()) {
#if ORACLE_MUTANT == 6  // mutant: the rule's ==/!= filters are ignored
        for (const Filter& f : std::vector<Filter>()) {
#else
        for (const Filter& f : r.filters) {
#endif
          uint32_t x, y;
          if (!eval_expr(f.a, val, x) || !eval_expr(f.b, val, y)) return;
          if (!compare_u32(f.cmp, x, y)) return;
        }
        Tuple h{};
        for (size_t c = 0; c < r.head.args.size(); c++) {
          if (!eval_expr(r.head_expr[c], val, h[c])) return;
          if (r.head_expr[c].op && h[c] == 0xFFFFFFFFu) return;
        }
#if ORACLE_MUTANT == 11  // mutant: the first two head columns are transposed
        if (r.head.args.size() >= 2) std::swap(h[0], h[1]);
#endif
        emit(h, tags);
        return;
      }
      const Atom& a = r.body[j];
      Key k;
      for (int c : bound_cols[j]) k.push_back(a.args[c].is_var ? val[a.args[c].value] : a.args[c].value);
      auto it = index[j].find(k);
      if (it == index[j].end()) return;
      for (auto* f : it->second) {
        std::vector<int> newly;
        bool ok = true;
        for (size_t c = 0; c < a.args.size() && ok; c++) {
          const Term& t = a.args[c];
          if (!t.is_var) continue;  // constants were part of the index key
          if (bound[t.value]) {
#if ORACLE_MUTANT != 7  // mutant 7: a variable bound earlier is not compared
            if (val[t.value] != f->first[c]) ok = false;
#endif
          } else {
            bound[t.value] = 1;
            val[t.value] = f->first[c];
            newly.push_back((int)t.value);
          }
        }
        if (ok) {
          tags[j] = &f->second;
          rec(j + 1);
        }
        for (int v : newly) bound[v] = 0;
      }
    };
    rec(0);
  }

  // Runs the strata in order, each to its fixpoint (Algorithm 1); max_iters
  // bounds the iterations of all strata together.  Returns 0 on fixpoint, -2
  // when max_iters iterations did not reach it.
  int run(uint32_t max_iters) {
#if ORACLE_MUTANT == 19  // mutant: one loop over every rule, strata ignored
    std::vector<std::vector<size_t>> strata(1);
    for (size_t i = 0; i < rules.size(); i++) strata[0].push_back(i);
#else
    const std::vector<std::vector<size_t>> strata = stratify(rules);
#endif
    uint32_t used = 0;
    for (const auto& stratum : strata) {
      const int rc = run_stratum(stratum, max_iters, used);
      if (rc) return rc;
    }
    return 0;
  }

  // One stratum: iterate its rules over the whole database until an iteration
  // changes nothing.  `used` counts the iterations run so far.
  int run_stratum(const std::vector<size_t>& stratum, uint32_t max_iters, uint32_t& used) {
#if ORACLE_MUTANT == 9  // mutant: max-min keeps the first tag of a key (key policy)
    const bool key_policy = (sr == ADD_MULT || sr == DIFF_ADD_MULT || sr == MAX_MIN);
#else
    const bool key_policy = (sr == ADD_MULT || sr == DIFF_ADD_MULT);
#endif
    for (uint32_t it = 0; used < max_iters; it++) {
      used++;
      std::map<std::string, std::map<Tuple, Acc>> derived;
      for (size_t ri : stratum) {
        const Rule& r = rules[ri];
        auto& out = derived[r.head.rel];
        const Relation* existing = nullptr;
        auto e = db.find(r.head.rel);
        if (e != db.end()) existing = &e->second;
        groundings(r, [&](const Tuple& h, const std::vector<const Tag*>& body) {
          Acc& acc = out[h];
          if (key_policy && existing && existing->count(h)) {
            acc.any = true;  // key already known: its tag is not recomputed
            return;
          }
          Tag g = *body[0];
          for (size_t j = 1; j < body.size(); j++) g = otimes(sr, g, *body[j]);
          acc_add(sr, acc, g);
        });
      }
      bool changed = false;
      for (auto& rel : derived) {
        Relation& R = db[rel.first];
        for (auto& kv : rel.second) {
          auto f = R.find(kv.first);
          if (f == R.end()) {
            R[kv.first] = acc_value(sr, kv.second);
            changed = true;
          } else if (!key_policy) {
            Acc merged;
            acc_add(sr, merged, f->second);
            acc_add(sr, merged, acc_value(sr, kv.second));
            Tag nv = acc_value(sr, merged);
            if (!tag_equal(sr, nv, f->second)) {
              f->second = nv;
              changed = true;
            }
          }
        }
      }
      iterations = (int)used;
#if ORACLE_MUTANT == 8  // mutant: stops after the second iteration
      if (it == 1) return 0;
#endif
      if (!changed) return 0;
    }
    return -2;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// C interface used by the Python test helpers
// ---------------------------------------------------------------------------
struct orc_input {
  std::string name;
  uint32_t arity;
  uint64_t base_id;  // input-fact id of row 0
  uint64_t n;
};

struct orc_result {
  int semiring;
  int iterations = 0;
  std::vector<orc_input> inputs;
  // relation -> sample -> sorted facts
  std::map<std::string, uint32_t> arity;
  std::map<std::string, std::map<uint32_t, Relation>> out;
  std::vector<double> prob;  // top-1-proofs: input-fact id -> probability
  uint64_t ties = 0;
};

extern "C" {

const char* orc_error(void) { return g_err.c_str(); }

int orc_run(const char* program, int semiring, int n_inputs, const char* const* names, const uint32_t* arities,
            const uint64_t* nrows, const uint32_t* const* cols, const double* const* tags,
            const uint32_t* const* samples, uint32_t max_iters, orc_result** result) {
  g_err.clear();
  if (!program || !result || semiring < 0 || semiring > 6 || n_inputs < 0) {
    g_err = "bad argument";
    return -3;
  }
  std::vector<Rule> rules;
  Parser p(program);
  if (!p.program(rules)) {
    g_err = "parse error near offset " + std::to_string(p.i);
    return -1;
  }
  auto* res = new orc_result();
  res->semiring = semiring;
  for (auto& r : rules) {
    res->arity[r.head.rel] = (uint32_t)r.head.args.size();
    for (auto& a : r.body) res->arity[a.rel] = (uint32_t)a.args.size();
  }
  // split loaded facts by sample; duplicates merged with (+)
  std::map<uint32_t, std::map<std::string, std::map<Tuple, Acc>>> loaded;
  uint64_t base = 0;
  g_prob.clear();
  g_proof_overflow = false;
  g_ties = 0;
  for (int k = 0; k < n_inputs; k++) base += nrows[k];
  if (is_top1(semiring)) g_prob.assign(base, 1.0);
  base = 0;
  for (int k = 0; k < n_inputs; k++) {
    if (arities[k] < 1 || arities[k] > (uint32_t)kMaxArity) {
      delete res;
      g_err = "bad arity";
      return -3;
    }
    res->inputs.push_back({names[k], arities[k], base, nrows[k]});
    res->arity[names[k]] = arities[k];
    for (uint64_t r = 0; r < nrows[k]; r++) {
      Tuple t{};
      for (uint32_t c = 0; c < arities[k]; c++) t[c] = cols[k][c * nrows[k] + r];
#if ORACLE_MUTANT == 10  // mutant: sample ids are ignored, so samples join
      uint32_t s = 0;
#else
      uint32_t s = samples && samples[k] ? samples[k][r] : 0;
#endif
      Tag g;
      g.v = tags && tags[k] ? tags[k][r] : 1.0;
      if (semiring == UNIT) g.v = 1.0;
      const bool differentiable = tags && tags[k];
      if (semiring == DIFF_MAX_MIN && differentiable) g.id = (uint32_t)(base + r);
      if (semiring == DIFF_ADD_MULT && differentiable) g.d[(uint32_t)(base + r)] = 1.0;
      if (is_top1(semiring) && differentiable) {
        g_prob[base + r] = g.v;
        g.proof.push_back((uint32_t)(base + r));
        g.v = proof_prob(g.proof);
      }
      acc_add(semiring, loaded[s][names[k]][t], g);
    }
    base += nrows[k];
  }
  if (loaded.empty()) loaded[0];
  if (g_proof_overflow) {  // a loaded proof alone is longer than the cap
    delete res;
    g_err = "a proof is longer than the proof cap";
    return -5;
  }
  // Samples never join, so each one is its own fixpoint; they run on separate
  // threads (one sample at a time per thread), and the results are gathered
  // in sample order, as a loop over the samples would produce them.
  struct SampleRun {
    uint32_t sample;
    std::map<std::string, std::map<Tuple, Acc>>* facts;
    Database db;
    int rc = 0, iterations = 0;
    bool overflow = false;
    uint64_t ties = 0;
  };
  const uint64_t load_ties = g_ties;  // ties met while merging duplicate loaded rows
  std::vector<SampleRun> runs;
  for (auto& smp : loaded) runs.push_back({smp.first, &smp.second, {}, 0, 0, false, 0});
  size_t next = 0;
  std::mutex mu;
  auto worker = [&]() {
    for (;;) {
      size_t i;
      {
        std::lock_guard<std::mutex> lock(mu);
        if (next >= runs.size()) return;
        i = next++;
      }
      SampleRun& sr = runs[i];
      g_proof_overflow = false;
      g_ties = 0;
      Engine e(semiring, rules);
      for (auto& rel : *sr.facts)
        for (auto& kv : rel.second) e.db[rel.first][kv.first] = acc_value(semiring, kv.second);
      sr.rc = e.run(max_iters);
      sr.iterations = e.iterations;
      sr.overflow = g_proof_overflow;
      sr.ties = g_ties;
      sr.db = std::move(e.db);
    }
  };
  const size_t n_threads = std::min<size_t>(runs.size(), std::max(1u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (size_t t = 1; t < n_threads; t++) {
    try {
      pool.emplace_back(worker);
    } catch (const std::system_error&) {
      break;  // no more threads: the ones started and this one share the samples
    }
  }
  worker();
  for (auto& t : pool) t.join();
  int max_it = 0;
  uint64_t ties = load_ties;
  for (auto& sr : runs) {
    if (sr.overflow) {
      delete res;
      g_err = "a proof is longer than the proof cap";
      return -5;
    }
    if (sr.rc != 0) {
      delete res;
      g_err = "max_iters reached";
      return sr.rc;
    }
    max_it = std::max(max_it, sr.iterations);
    ties += sr.ties;
    for (auto& rel : sr.db) res->out[rel.first][sr.sample] = std::move(rel.second);
  }
  res->iterations = max_it;
  res->prob = g_prob;
  res->ties = ties;
  *result = res;
  return 0;
}

int orc_iterations(const orc_result* r) { return r ? r->iterations : -1; }

// top-1-proofs: the proof cap of later runs (default 300)
void orc_set_proof_cap(uint32_t cap) { g_proof_cap = cap; }

// top-1-proofs: equally likely different proofs met by (+) during the run
uint64_t orc_ties(const orc_result* r) { return r ? r->ties : 0; }

// top-1-proofs: the proofs of `rel` in read order, as per-fact lengths and the
// concatenated ascending input-fact ids; returns the total number of ids (call
// with null pointers to size the buffers).
int64_t orc_read_proofs(const orc_result* r, const char* rel, uint32_t* lens, uint32_t* ids) {
  auto it = r->out.find(rel);
  if (it == r->out.end()) return 0;
  int64_t i = 0, w = 0;
  for (auto& s : it->second)
    for (auto& kv : s.second) {
      if (lens) lens[i] = (uint32_t)kv.second.proof.size();
      for (uint32_t id : kv.second.proof) {
        if (ids) ids[w] = id;
        w++;
      }
      i++;
    }
  return w;
}

int64_t orc_size(const orc_result* r, const char* rel) {
  auto it = r->out.find(rel);
  if (it == r->out.end()) return r->arity.count(rel) ? 0 : -1;
  int64_t n = 0;
  for (auto& s : it->second) n += (int64_t)s.second.size();
  return n;
}

int orc_arity(const orc_result* r, const char* rel) {
  auto it = r->arity.find(rel);
  return it == r->arity.end() ? -1 : (int)it->second;
}

// cols: arity x n column-major; tags, samples nullable.  Sorted by (sample, cols).
int orc_read(const orc_result* r, const char* rel, uint32_t* cols, double* tags, uint32_t* samples) {
  auto it = r->out.find(rel);
  if (it == r->out.end()) return 0;
  uint32_t ar = r->arity.at(rel);
  int64_t n = orc_size(r, rel);
  int64_t i = 0;
  for (auto& s : it->second)
    for (auto& kv : s.second) {
      for (uint32_t c = 0; c < ar; c++) cols[c * n + i] = kv.first[c];
      if (tags) tags[i] = kv.second.v;
      if (samples) samples[i] = s.first;
      i++;
    }
  return 0;
}

// For diff-max-min: the input-fact id (global row index over all inputs in
// load order) that bounds each output tag, or 0xFFFFFFFF.
int orc_read_ids(const orc_result* r, const char* rel, uint32_t* ids) {
  auto it = r->out.find(rel);
  if (it == r->out.end()) return 0;
  int64_t i = 0;
  for (auto& s : it->second)
    for (auto& kv : s.second) ids[i++] = kv.second.id;
  return 0;
}

// Vector-Jacobian product: grad_in[k][row] += sum_o grad_out[o] * d tag_o / d p_(k,row)
// with o running over `rel` in read order.  Only for the diff semirings.
int orc_vjp(const orc_result* r, const char* rel, const double* grad_out, double* const* grad_in) {
  if (r->semiring != DIFF_MAX_MIN && r->semiring != DIFF_ADD_MULT && r->semiring != DIFF_TOP1) return -4;
  auto it = r->out.find(rel);
  if (it == r->out.end()) return 0;
  auto deposit = [&](uint32_t id, double g) {
    for (size_t k = 0; k < r->inputs.size(); k++) {
      const orc_input& in = r->inputs[k];
      if (id >= in.base_id && id < in.base_id + in.n) {
        if (grad_in[k]) grad_in[k][id - in.base_id] += g;
        return;
      }
    }
  };
  int64_t i = 0;
  for (auto& s : it->second)
    for (auto& kv : s.second) {
      double g = grad_out[i++];
      if (r->semiring == DIFF_MAX_MIN) {
        if (kv.second.id != kNoId) deposit(kv.second.id, g);
      } else if (r->semiring == DIFF_TOP1) {
        // d prod_j p_j / d p_i = product of the other facts' probabilities
        const std::vector<uint32_t>& P = kv.second.proof;
        for (size_t a = 0; a < P.size(); a++) {
          double others = 1.0;
          for (size_t b = 0; b < P.size(); b++)
            if (b != a) others *= r->prob[P[b]];
          deposit(P[a], g * others);
        }
      } else {
        for (auto& d : kv.second.d) deposit(d.first, g * d.second);
      }
    }
  return 0;
}

void orc_free(orc_result* r) { delete r; }

}  // extern "C"
