// Rule text -> RuleAst (engine-side parser; range-restriction checks).
#include <cctype>
#include <cstring>

#include "engine.h"

namespace {

enum TokKind { T_IDENT, T_NUM, T_LPAR, T_RPAR, T_COMMA, T_DOT, T_IF, T_NE, T_EQ, T_END };
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
    r.head = atom();
    expect(T_IF, "':-'");
    for (;;) {
      if (peek().k == T_IDENT && peek(1).k == T_LPAR) {
        r.body.push_back(atom());
      } else {
        FilterAst f;
        f.a = term();
        if (peek().k == T_NE) f.eq = false;
        else if (peek().k == T_EQ) f.eq = true;
        else fail("expected '!=' or '=='");
        p++;
        f.b = term();
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
