// KXMECH 1 reader and validator for the kx library.
//
// The file is line oriented: a keyword, then whitespace-separated fields.
// Doubles are written in shortest round-trip form and read with strtod, so
// the constants folded into the generated kernels are bit-identical to the
// file.  Validation covers index ranges, positive molecular weights,
// physical parameter ranges and atom balance of every reaction.
#include <cerrno>
#include <cmath>
#include <cstdlib>
#include <fstream>
#include <sstream>

#include "kx_internal.h"

namespace kx {
namespace {

struct Reader {
  std::vector<std::string> tok;
  size_t pos = 0;
  std::string err;
  bool ok = true;

  void fail(const std::string& e) {
    if (ok) err = e;
    ok = false;
  }
  std::string word() {
    if (pos >= tok.size()) { fail("unexpected end of record"); return ""; }
    return tok[pos++];
  }
  double real() {
    std::string s = word();
    if (!ok) return 0.0;
    char* end = nullptr;
    errno = 0;
    double v = std::strtod(s.c_str(), &end);
    if (end == s.c_str() || *end != '\0' || errno == ERANGE || !std::isfinite(v)) fail("bad number '" + s + "'");
    return v;
  }
  long integer() {
    std::string s = word();
    if (!ok) return 0;
    char* end = nullptr;
    long v = std::strtol(s.c_str(), &end, 10);
    if (end == s.c_str() || *end != '\0') fail("bad integer '" + s + "'");
    return v;
  }
};

bool in_range(long v, long hi) { return v >= 0 && v < hi; }

}  // namespace

kx_status parse_mechanism(const std::string& path, Mechanism& m, std::string& err) {
  std::ifstream in(path);
  if (!in) { err = "cannot open " + path; return KX_ERR_IO; }
  std::string line;
  int lineno = 0;
  bool header = false, done = false;
  int declared_nr = -1;
  Reaction* cur = nullptr;
  while (std::getline(in, line)) {
    ++lineno;
    Reader r;
    std::istringstream ss(line);
    for (std::string w; ss >> w;) r.tok.push_back(w);
    if (r.tok.empty() || r.tok[0][0] == '#') continue;
    auto bad = [&](const std::string& e) {
      err = path + ":" + std::to_string(lineno) + ": " + e;
      return KX_ERR_PARSE;
    };
    const std::string key = r.word();
    if (!header) {
      if (key != "KXMECH" || r.word() != "1") return bad("expected header 'KXMECH 1'");
      header = true;
      continue;
    }
    if (done) return bad("data after end_mechanism");
    if (key == "name") {
      m.name = r.word();
    } else if (key == "elements") {
      long ne = r.integer();
      if (ne <= 0 || ne > 64) return bad("bad element count");
      for (long e = 0; e < ne; ++e) m.elements.push_back(r.word());
    } else if (key == "species") {
      long ns = r.integer();
      if (ns <= 0 || ns > 4096 || m.elements.empty()) return bad("bad species count (or elements missing)");
      m.ns = (int)ns;
      m.species.assign(ns, "");
      m.W.assign(ns, 0.0);
      m.comp.assign(ns * m.elements.size(), 0);
      m.inert.assign(ns, 0);
      m.Tlow.assign(ns, 0.0); m.Tmid.assign(ns, 0.0); m.Thigh.assign(ns, 0.0);
      m.a_lo.assign(7 * ns, 0.0); m.a_hi.assign(7 * ns, 0.0);
      m.eta.assign(5 * ns, 0.0); m.lam.assign(5 * ns, 0.0);
      m.dif.assign((size_t)5 * ns * ns, 0.0);
    } else if (key == "species_data") {
      long k = r.integer();
      if (!in_range(k, m.ns)) return bad("species index out of range");
      m.species[k] = r.word();
      m.W[k] = r.real();
      m.inert[k] = (char)(r.integer() != 0);
      for (size_t e = 0; e < m.elements.size(); ++e) {
        long c = r.integer();
        if (c < 0) return bad("negative atom count");
        m.comp[k * m.elements.size() + e] = (int)c;
      }
      if (r.ok && !(m.W[k] > 0.0)) return bad("molecular weight must be positive");
    } else if (key == "nasa") {
      long k = r.integer();
      if (!in_range(k, m.ns)) return bad("species index out of range");
      m.Tlow[k] = r.real(); m.Tmid[k] = r.real(); m.Thigh[k] = r.real();
      for (int j = 0; j < 7; ++j) m.a_lo[7 * k + j] = r.real();
      for (int j = 0; j < 7; ++j) m.a_hi[7 * k + j] = r.real();
      if (r.ok && !(m.Tmid[k] > 0.0)) return bad("NASA mid temperature must be positive");
    } else if (key == "transport_fit") {
      const std::string v = r.word();
      if (v == "ln") m.fit_direct = false;
      else if (v == "direct") m.fit_direct = true;
      else return bad("transport_fit must be ln or direct");
    } else if (key == "eta" || key == "lambda") {
      long k = r.integer();
      if (!in_range(k, m.ns)) return bad("species index out of range");
      for (int j = 0; j < 5; ++j) (key == "eta" ? m.eta : m.lam)[5 * k + j] = r.real();
    } else if (key == "diff") {
      long a = r.integer(), b = r.integer();
      if (!in_range(a, m.ns) || !in_range(b, m.ns)) return bad("species index out of range");
      for (int j = 0; j < 5; ++j) {
        double v = r.real();
        m.dif[5 * ((size_t)a * m.ns + b) + j] = v;
        m.dif[5 * ((size_t)b * m.ns + a) + j] = v;
      }
    } else if (key == "reactions") {
      declared_nr = (int)r.integer();
      if (declared_nr < 0) return bad("bad reaction count");
    } else if (key == "reaction") {
      r.integer();
      std::string kind = r.word();
      Reaction rx;
      if (kind == "elementary") rx.kind = Kind::Elementary;
      else if (kind == "three_body") rx.kind = Kind::ThreeBody;
      else if (kind == "falloff") rx.kind = Kind::Falloff;
      else if (kind == "chem_act") rx.kind = Kind::ChemAct;
      else if (kind == "plog") rx.kind = Kind::Plog;
      else return bad("unknown reaction kind '" + kind + "'");
      rx.reversible = r.integer() != 0;
      m.rx.push_back(rx);
      cur = &m.rx.back();
    } else if (key == "reactants" || key == "products") {
      if (!cur) return bad("record outside a reaction");
      long n = r.integer();
      if (n < 1 || n > 8) return bad("bad species count in reaction side");
      for (long j = 0; j < n; ++j) {
        long k = r.integer(), nu = r.integer();
        if (!in_range(k, m.ns) || nu < 1 || nu > 3) return bad("bad species/coefficient in reaction");
        (key == "reactants" ? cur->reac : cur->prod).push_back({(int)k, (int)nu});
      }
    } else if (key == "rate" || key == "rate_low") {
      if (!cur) return bad("record outside a reaction");
      Arrh a{r.real(), r.real(), r.real()};
      if (r.ok && !(a.A >= 0.0)) return bad("negative pre-exponential factor");
      if (key == "rate") cur->k = a;
      else { cur->k0 = a; cur->has_k0 = true; }
    } else if (key == "third_body") {
      if (!cur) return bad("record outside a reaction");
      cur->default_eff = r.real();
      long n = r.integer();
      for (long j = 0; j < n; ++j) {
        long k = r.integer();
        double a = r.real();
        if (!in_range(k, m.ns) || a < 0.0) return bad("bad efficiency");
        cur->eff.push_back({(int)k, a});
      }
    } else if (key == "collider") {
      if (!cur) return bad("record outside a reaction");
      long k = r.integer();
      if (!in_range(k, m.ns)) return bad("collider out of range");
      cur->collider = (int)k;
    } else if (key == "troe") {
      if (!cur) return bad("record outside a reaction");
      cur->blend = Blend::Troe;
      for (int j = 0; j < 4; ++j) cur->troe[j] = r.real();
      if (r.ok && (cur->troe[1] == 0.0 || cur->troe[2] == 0.0)) return bad("Troe T*** and T* must be nonzero");
    } else if (key == "sri") {
      if (!cur) return bad("record outside a reaction");
      cur->blend = Blend::Sri;
      for (int j = 0; j < 5; ++j) cur->sri[j] = r.real();
      if (r.ok && cur->sri[2] == 0.0) return bad("SRI c must be nonzero");
    } else if (key == "plog") {
      if (!cur) return bad("record outside a reaction");
      long n = r.integer();
      if (n < 1 || n > 64) return bad("bad PLOG count");
      for (long j = 0; j < n; ++j) {
        std::array<double, 4> e{r.real(), r.real(), r.real(), r.real()};
        if (r.ok && !(e[0] > 0.0 && e[1] > 0.0)) return bad("PLOG pressure and A must be positive");
        if (!cur->plog.empty() && r.ok && !(e[0] > cur->plog.back()[0])) return bad("PLOG pressures must ascend");
        cur->plog.push_back(e);
      }
    } else if (key == "end") {
      cur = nullptr;
    } else if (key == "end_mechanism") {
      done = true;
    } else {
      return bad("unknown record '" + key + "'");
    }
    if (!r.ok) return bad(r.err);
  }
  if (!header) { err = path + ": empty file"; return KX_ERR_PARSE; }
  if (!done) { err = path + ": missing end_mechanism"; return KX_ERR_PARSE; }
  if (m.ns == 0) { err = path + ": no species"; return KX_ERR_PARSE; }
  if (declared_nr >= 0 && declared_nr != m.nr()) { err = path + ": reaction count mismatch"; return KX_ERR_PARSE; }
  const size_t ne = m.elements.size();
  for (int k = 0; k < m.ns; ++k)
    if (m.species[k].empty() || !(m.Tmid[k] > 0.0)) { err = path + ": species " + std::to_string(k) + " incomplete"; return KX_ERR_PARSE; }
  for (int i = 0; i < m.nr(); ++i) {
    const Reaction& rx = m.rx[i];
    if (rx.reac.empty() || rx.prod.empty()) { err = "reaction " + std::to_string(i) + " has an empty side"; return KX_ERR_PARSE; }
    if ((rx.kind == Kind::Falloff || rx.kind == Kind::ChemAct) && !rx.has_k0) {
      err = "reaction " + std::to_string(i) + ": falloff without rate_low"; return KX_ERR_PARSE;
    }
    if (rx.kind == Kind::Plog && rx.plog.empty()) { err = "reaction " + std::to_string(i) + ": PLOG without table"; return KX_ERR_PARSE; }
    for (size_t e = 0; e < ne; ++e) {
      long bal = 0;
      for (auto& s : rx.reac) bal -= (long)s.second * m.comp[s.first * ne + e];
      for (auto& s : rx.prod) bal += (long)s.second * m.comp[s.first * ne + e];
      if (bal != 0) {
        err = "reaction " + std::to_string(i) + " does not conserve element " + m.elements[e];
        return KX_ERR_UNBALANCED;
      }
    }
  }
  return KX_OK;
}

}  // namespace kx
