// Rule text -> RuleAst (engine-side parser; range-restriction checks).
#include <cctype>
#include <cstring>

#include "engine.h"

namespace {

enum TokKind {
  T_IDENT, T_NUM, T_LPAR, T_RPAR, T_COMMA, T_DOT, T_IF, T_NE, T_EQ, T_LT, T_LE, T_GT, T_GE, T_PLUS, T_MINUS, T_STAR,
  T_SLASH, T_END
};
struct Tok {
  TokKind k;
  std::string s;
  unsigned long long num = 0;
  size_t at = 0;
};

std::vector<Tok> lex(const char* text) {
  std::vector<Tok> out;
  size_t i = 0, n = std::strlen(text);
  while (i < n) {
    char c = text[i];
    if (std::isspace((unsigned char)c)) { i++; continue; }
    if (c == '%' || c == '#' || (c == '/' && i + 1 < n && text[i + 1] == '/')) {
      while (i < n && text[i] != '\n') i++;
      continue;
    }
    Tok t;
    t.at = i;
    if (std::isalpha((unsigned char)c) || c == '_') {
      size_t j = i;
      while (j < n && (std::isalnum((unsigned char)text[j]) || text[j] == '_')) j++;
      t.k = T_IDENT;
      t.s.assign(text + i, j - i);
      i = j;
    } else if (std::isdigit((unsigned char)c)) {
      size_t j = i;
      unsigned long long v = 0;
      while (j < n && std::isdigit((unsigned char)text[j])) {
        v = v * 10 + (unsigned)(text[j] - '0');
        if (v > 0xFFFFFFFEull) throw LobError(LOB_E_PARSE, "constant too large at offset " + std::to_string(i));
        j++;
      }
      t.k = T_NUM;
      t.num = v;
      i = j;
    } else if (c == '(') { t.k = T_LPAR; i++; }
    else if (c == ')') { t.k = T_RPAR; i++; }
    else if (c == ',') { t.k = T_COMMA; i++; }
    else if (c == '.') { t.k = T_DOT; i++; }
    else if (c == ':' && i + 1 < n && text[i + 1] == '-') { t.k = T_IF; i += 2; }
    else if (c == '!' && i + 1 < n && text[i + 1] == '=') { t.k = T_NE; i += 2; }
    else if (c == '=' && i + 1 < n && text[i + 1] == '=') { t.k = T_EQ; i += 2; }
    else if (c == '<' && i + 1 < n && text[i + 1] == '=') { t.k = T_LE; i += 2; }
    else if (c == '>' && i + 1 < n && text[i + 1] == '=') { t.k = T_GE; i += 2; }
    else if (c == '<') { t.k = T_LT; i++; }
    else if (c == '>') { t.k = T_GT; i++; }
    else if (c == '+') { t.k = T_PLUS; i++; }
    else if (c == '-') { t.k = T_MINUS; i++; }
    else if (c == '*') { t.k = T_STAR; i++; }
    else if (c == '/') { t.k = T_SLASH; i++; }
    else throw LobError(LOB_E_PARSE, std::string("unexpected character '") + c + "' at offset " + std::to_string(i));
    out.push_back(t);
  }
  Tok e;
  e.k = T_END;
  e.at = n;
  out.push_back(e);
  return out;
}

struct RuleParser {
  const lob_engine& eng;
  std::vector<Tok> toks;
  size_t p = 0;
  RuleAst r;
  std::map<std::string, u32> slots;

  RuleParser(const lob_engine& e, const char* text) : eng(e), toks(lex(text)) { r.text = text; }

  [[noreturn]] void fail(const std::string& what) {
    throw LobError(LOB_E_PARSE, what + " at offset " + std::to_string(toks[p].at));
  }
  const Tok& peek(int k = 0) const { return toks[std::min(p + k, toks.size() - 1)]; }
  void expect(TokKind k, const char* what) {
    if (peek().k != k) fail(std::string("expected ") + what);
    p++;
  }
  Term term() {
    Term t;
    if (peek().k == T_NUM) {
      t.var = false;
      t.v = (u32)peek().num;
      p++;
      return t;
    }
    if (peek().k != T_IDENT) fail("expected a variable or a constant");
    const std::string& name = peek().s;
    auto it = slots.find(name);
    if (it == slots.end()) {
      if (slots.size() >= (size_t)kMaxSlots) throw LobError(LOB_E_ARG, "rule has more than 16 variables");
      it = slots.emplace(name, (u32)slots.size()).first;
      r.var_names.push_back(name);
    }
    t.var = true;
    t.v = it->second;
    p++;
    return t;
  }
  // Expressions (Sec. 5.2): expr := product (('+' | '-') product)*,
  // product := primary (('*' | '/') primary)*, primary := term | '(' expr ')'.
  // Parsed into a small tree, then emitted in postfix order as bytecode.
  struct Node {
    int op = -1;  // -1: leaf; else a BcOp
    Term leaf;
    int l = -1, r = -1;
  };
  std::vector<Node> nodes;
  int primary() {
    if (peek().k == T_LPAR) {
      p++;
      const int e = expr();
      expect(T_RPAR, "')'");
      return e;
    }
    Node n;
    n.leaf = term();
    nodes.push_back(n);
    return (int)nodes.size() - 1;
  }
  int binary(int op, int l, int r) {
    Node n;
    n.op = op;
    n.l = l;
    n.r = r;
    nodes.push_back(n);
    return (int)nodes.size() - 1;
  }
  int product() {
    int e = primary();
    while (peek().k == T_STAR || peek().k == T_SLASH) {
      const int op = peek().k == T_STAR ? BC_MUL : BC_DIV;
      p++;
      e = binary(op, e, primary());
    }
    return e;
  }
  int expr() {
    int e = product();
    while (peek().k == T_PLUS || peek().k == T_MINUS) {
      const int op = peek().k == T_PLUS ? BC_ADD : BC_SUB;
      p++;
      e = binary(op, e, product());
    }
    return e;
  }
  // postfix code of node e; returns its stack depth and collects its variables
  int emit(int e, std::vector<BcIns>& code, std::vector<u32>& vars) {
    const Node& n = nodes[e];
    BcIns I{};
    if (n.op < 0) {
      I.op = n.leaf.var ? BC_VAR : BC_CONST;
      I.slot = (uint8_t)(n.leaf.var ? n.leaf.v : 0);
      I.imm = n.leaf.var ? 0 : n.leaf.v;
      if (n.leaf.var) vars.push_back(n.leaf.v);
      code.push_back(I);
      return 1;
    }
    const int dl = emit(n.l, code, vars);
    const int dr = emit(n.r, code, vars);
    I.op = (uint8_t)n.op;
    code.push_back(I);
    return std::max(dl, 1 + dr);
  }
  // one program computing node e (then `tail_op`, a comparison, when >= 0 on
  // two nodes); returns its 1-based program number
  int program(int e, int e2, int cmp, std::vector<u32>& vars) {
    std::vector<BcIns> code;
    int depth = emit(e, code, vars);
    if (e2 >= 0) {
      depth = std::max(depth, 1 + emit(e2, code, vars));
      BcIns I{};
      I.op = (uint8_t)cmp;
      code.push_back(I);
    }
    if (depth > kBcStack) fail("expression too deep for the bytecode stack");
    if (r.code.size() + code.size() > (size_t)kMaxCode || r.progs.size() >= (size_t)kMaxProgs)
      fail("rule has too much arithmetic (at most 64 instructions in 16 expressions)");
    r.progs.emplace_back((int)r.code.size(), (int)code.size());
    r.code.insert(r.code.end(), code.begin(), code.end());
    return (int)r.progs.size();
  }
  AtomAst head_atom() {
    AtomAst a;
    if (peek().k != T_IDENT) fail("expected a relation name");
    auto it = eng.rel_ids.find(peek().s);
    if (it == eng.rel_ids.end()) throw LobError(LOB_E_UNKNOWN_REL, "unknown relation '" + peek().s + "'");
    a.rel = it->second;
    p++;
    expect(T_LPAR, "'('");
    for (;;) {
      const int e = expr();
      if (nodes[e].op < 0) {
        a.args.push_back(nodes[e].leaf);
        r.head_prog.push_back(0);
      } else {
        Term t;  // placeholder: the column is computed
        a.args.push_back(t);
        r.head_prog.push_back(program(e, -1, 0, r.head_vars));
      }
      if (peek().k != T_COMMA) break;
      p++;
    }
    expect(T_RPAR, "')'");
    if (a.args.size() != eng.rels[a.rel].arity)
      throw LobError(LOB_E_ARG, "relation '" + eng.rels[a.rel].name + "' has arity " +
                                    std::to_string(eng.rels[a.rel].arity) + ", used with " +
                                    std::to_string(a.args.size()) + " arguments");
    return a;
  }
  AtomAst atom() {
    AtomAst a;
    if (peek().k != T_IDENT) fail("expected a relation name");
    auto it = eng.rel_ids.find(peek().s);
    if (it == eng.rel_ids.end()) throw LobError(LOB_E_UNKNOWN_REL, "unknown relation '" + peek().s + "'");
    a.rel = it->second;
    p++;
    expect(T_LPAR, "'('");
    a.args.push_back(term());
    while (peek().k == T_COMMA) {
      p++;
      a.args.push_back(term());
    }
    expect(T_RPAR, "')'");
    if (a.args.size() != eng.rels[a.rel].arity)
      throw LobError(LOB_E_ARG, "relation '" + eng.rels[a.rel].name + "' has arity " +
                                    std::to_string(eng.rels[a.rel].arity) + ", used with " +
                                    std::to_string(a.args.size()) + " arguments");
    return a;
  }
  RuleAst parse() {
    r.head = head_atom();
    expect(T_IF, "':-'");
    for (;;) {
      if (peek().k == T_IDENT && peek(1).k == T_LPAR) {
        r.body.push_back(atom());
      } else {
        FilterAst f;
        const int a = expr();
        int cmp;
        switch (peek().k) {
          case T_NE: cmp = BC_NE; break;
          case T_EQ: cmp = BC_EQ; break;
          case T_LT: cmp = BC_LT; break;
          case T_LE: cmp = BC_LE; break;
          case T_GT: cmp = BC_GT; break;
          case T_GE: cmp = BC_GE; break;
          default: fail("expected a comparison (==, !=, <, <=, >, >=)");
        }
        p++;
        const int b = expr();
        if ((cmp == BC_EQ || cmp == BC_NE) && nodes[a].op < 0 && nodes[b].op < 0) {
          f.a = nodes[a].leaf;  // plain (in)equality of two terms: no bytecode
          f.b = nodes[b].leaf;
          f.eq = cmp == BC_EQ;
        } else {
          f.prog = program(a, b, cmp, f.vars);
        }
        r.filters.push_back(f);
      }
      if (peek().k == T_COMMA) { p++; continue; }
      break;
    }
    expect(T_DOT, "'.'");
    if (peek().k != T_END) fail("one rule per call: text after '.'");
    if (r.body.empty()) fail("rule without a body atom");
    if (r.body.size() > (size_t)kMaxArity) throw LobError(LOB_E_ARG, "rule has more than 8 body atoms");
    if (r.filters.size() > (size_t)kMaxFilters) throw LobError(LOB_E_ARG, "rule has more than 8 filters");
    // range restriction: every variable must occur in a body atom
    std::vector<char> bound(r.var_names.size(), 0);
    for (auto& a : r.body)
      for (auto& t : a.args)
        if (t.var) bound[t.v] = 1;
    for (auto& t : r.head.args)
      if (t.var && !bound[t.v])
        throw LobError(LOB_E_UNSAFE_RULE, "head variable '" + r.var_names[t.v] + "' does not occur in the body");
    for (u32 v : r.head_vars)
      if (!bound[v])
        throw LobError(LOB_E_UNSAFE_RULE, "head variable '" + r.var_names[v] + "' does not occur in the body");
    for (auto& f : r.filters)
      for (u32 v : f.vars)
        if (!bound[v])
          throw LobError(LOB_E_UNSAFE_RULE, "filter variable '" + r.var_names[v] + "' does not occur in a body atom");
    for (auto& f : r.filters)
      for (const Term* t : {&f.a, &f.b})
        if (t->var && !bound[t->v])
          throw LobError(LOB_E_UNSAFE_RULE, "filter variable '" + r.var_names[t->v] + "' does not occur in a body atom");
    return r;
  }
};

}  // namespace

RuleAst parse_rule(const lob_engine& e, const char* text) {
  RuleParser p(e, text);
  return p.parse();
}

bool valid_ident(const char* s) {
  if (!s || !(std::isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
  for (const char* c = s; *c; c++)
    if (!(std::isalnum((unsigned char)*c) || *c == '_')) return false;
  return true;
}
