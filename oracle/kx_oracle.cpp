// FP64 CPU oracle for the per-point chemistry source term, thermodynamic
// properties and mixture-averaged transport of KinetiX (arXiv 2411.02640,
// Appendix A).
//
// TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
// GPU kernels are checked against.  Only tests, the smoke check and the CPU
// baseline leg of the benchmark may load it.  It shares no code, header or
// table with the GPU library: it has its own mechanism-file reader and writes
// every formula out in the textbook order, point by point, in double
// precision, with no exponential sharing, no log-space rewriting and no
// reordering beyond what the equations state.  Build with -ffp-contract=off.
//
// Every function is a template over the scalar type so that the same
// formulas, evaluated on forward-mode dual numbers, give the dense Jacobian
// d(wdot)/d(T, Y) used to check the adjoint kernel.
//
// Readings where the paper is silent or garbled (documented with the design):
//   * "log" in the Troe and SRI blending is log10 (Eq. blend, Sec. A.2.2).
//   * The Troe display is read as log F = log Fcent / (1 + f^2),
//     f = (log Pr + c) / (n - d (log Pr + c)).
//   * Pr is floored at 1e-300 before its logarithm is taken.
//   * The T** term of Fcent is always included.
//   * Falloff: k_f is the blended constant k_inf Pr/(1+Pr) F and the modifier
//     c_i is 1, so the blending is not applied twice; chemically activated:
//     k_f = k_0 F/(1+Pr).
//   * The third body of a falloff reaction is the efficiency-weighted mixture
//     (or the named collider species).
//   * Concentrations C_k = (p/(R T)) (Y_k/W_k) / sum_j Y_j/W_j, so that the
//     rates are homogeneous of degree 0 in Y.
//   * NASA-7: the low block is used for T < Tmid, the high block otherwise.
//   * D_kj(T, p) = D_kj(T, 1 atm) p_atm / p; D_k falls back to D_kk when the
//     sum over the other species vanishes (a pure species).
//   * cp and h are mass-based mixture values: J/(kg K) and J/kg.
//   * PLOG outside the tabulated pressures uses the nearest end rate.
//   * Wilke's phi_kj uses (W_j/W_k)^(1/4) (the standard Wilke/Bird form);
//     the appendix prints (W_k/W_j)^(1/4).
// Units: SI with kmol (W in kg/kmol, C in kmol/m^3, wdot in kmol/(m^3 s)).

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>
#include <algorithm>

namespace {

const double R_U = 8314.46261815324;   // J/(kmol K)
const double P_ATM = 101325.0;         // Pa

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { double q = a.v / b.v; return Dual(q, (a.d - q * b.d) / b.v); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual log10(Dual a) { return Dual(std::log10(a.v), a.d / (a.v * std::log(10.0))); }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, 0.5 * a.d / s); }
inline Dual pow(Dual a, double b) { double p = std::pow(a.v, b); return Dual(p, b * std::pow(a.v, b - 1.0) * a.d); }
inline Dual pow(double a, Dual b) { double p = std::pow(a, b.v); return Dual(p, p * std::log(a) * b.d); }
inline Dual pow(Dual a, Dual b) { return exp(b * log(a)); }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }

using std::exp; using std::log; using std::log10; using std::sqrt; using std::pow;

// ---------------------------------------------------------------- mechanism
enum Kind { ELEMENTARY = 0, THREE_BODY = 1, FALLOFF = 2, CHEM_ACT = 3, PLOG = 4 };

struct Arr { double A = 0, beta = 0, E = 0; };

struct Rxn {
  int kind = ELEMENTARY;
  bool reversible = true;
  std::vector<std::pair<int, int>> reac, prod;   // (species, coefficient)
  Arr rate, low;
  double default_eff = 1.0;
  std::vector<std::pair<int, double>> eff;
  int collider = -1;
  bool troe = false, sri = false;
  double troe_p[4] = {0, 0, 0, 0};                // alpha, T***, T*, T**
  double sri_p[5] = {0, 0, 0, 1, 0};              // a, b, c, d, e
  std::vector<double> plog_p, plog_A, plog_b, plog_E;
};

struct Mech {
  int ns = 0, nr = 0;
  std::vector<double> W;
  std::vector<double> Tmid;
  std::vector<double> a_lo, a_hi;      // [ns][7]
  std::vector<double> eta, lam;        // [ns][5]
  std::vector<double> dif;             // [ns][ns][5]
  bool direct = false;                 // fits of eta, lambda and 1/D_kj themselves (else of their logs)
  std::vector<Rxn> rx;
};

bool parse(const char* path, Mech& m, std::string& err) {
  FILE* f = std::fopen(path, "r");
  if (!f) { err = "cannot open"; return false; }
  std::vector<std::vector<std::string>> lines;
  char buf[1 << 16];
  std::string cur;
  while (std::fgets(buf, sizeof buf, f)) {
    cur += buf;
    if (cur.empty() || cur.back() != '\n') continue;
    std::vector<std::string> t;
    char* save = nullptr;
    for (char* p = strtok_r(&cur[0], " \t\r\n", &save); p; p = strtok_r(nullptr, " \t\r\n", &save)) t.push_back(p);
    if (!t.empty() && t[0][0] != '#') lines.push_back(t);
    cur.clear();
  }
  std::fclose(f);
  if (lines.empty() || lines[0].size() < 2 || lines[0][0] != "KXMECH" || lines[0][1] != "1") { err = "bad header"; return false; }
  auto D = [](const std::string& s) { return std::strtod(s.c_str(), nullptr); };
  auto I = [](const std::string& s) { return (int)std::strtol(s.c_str(), nullptr, 10); };
  for (size_t li = 1; li < lines.size(); ++li) {
    auto& t = lines[li];
    const std::string& k = t[0];
    if (k == "species") {
      m.ns = I(t[1]);
      m.W.assign(m.ns, 0); m.Tmid.assign(m.ns, 0);
      m.a_lo.assign(7 * m.ns, 0); m.a_hi.assign(7 * m.ns, 0);
      m.eta.assign(5 * m.ns, 0); m.lam.assign(5 * m.ns, 0); m.dif.assign(5 * m.ns * m.ns, 0);
    } else if (k == "species_data") {
      m.W[I(t[1])] = D(t[3]);
    } else if (k == "nasa") {
      int s = I(t[1]);
      m.Tmid[s] = D(t[3]);
      for (int j = 0; j < 7; ++j) { m.a_lo[7 * s + j] = D(t[5 + j]); m.a_hi[7 * s + j] = D(t[12 + j]); }
    } else if (k == "transport_fit") {
      m.direct = t[1] == "direct";
    } else if (k == "eta" || k == "lambda") {
      int s = I(t[1]);
      for (int j = 0; j < 5; ++j) (k == "eta" ? m.eta : m.lam)[5 * s + j] = D(t[2 + j]);
    } else if (k == "diff") {
      int a = I(t[1]), b = I(t[2]);
      for (int j = 0; j < 5; ++j) { m.dif[5 * (a * m.ns + b) + j] = D(t[3 + j]); m.dif[5 * (b * m.ns + a) + j] = D(t[3 + j]); }
    } else if (k == "reaction") {
      Rxn r;
      const std::string& kind = t[2];
      r.kind = kind == "elementary" ? ELEMENTARY : kind == "three_body" ? THREE_BODY : kind == "falloff" ? FALLOFF
             : kind == "chem_act" ? CHEM_ACT : kind == "plog" ? PLOG : -1;
      if (r.kind < 0) { err = "unknown reaction kind " + kind; return false; }
      r.reversible = I(t[3]) != 0;
      m.rx.push_back(r);
    } else if (k == "reactants" || k == "products") {
      int n = I(t[1]);
      auto& v = (k == "reactants") ? m.rx.back().reac : m.rx.back().prod;
      for (int j = 0; j < n; ++j) v.push_back({I(t[2 + 2 * j]), I(t[3 + 2 * j])});
    } else if (k == "rate") {
      m.rx.back().rate = {D(t[1]), D(t[2]), D(t[3])};
    } else if (k == "rate_low") {
      m.rx.back().low = {D(t[1]), D(t[2]), D(t[3])};
    } else if (k == "third_body") {
      Rxn& r = m.rx.back();
      r.default_eff = D(t[1]);
      int n = I(t[2]);
      for (int j = 0; j < n; ++j) r.eff.push_back({I(t[3 + 2 * j]), D(t[4 + 2 * j])});
    } else if (k == "collider") {
      m.rx.back().collider = I(t[1]);
    } else if (k == "troe") {
      Rxn& r = m.rx.back(); r.troe = true;
      for (int j = 0; j < 4; ++j) r.troe_p[j] = D(t[1 + j]);
    } else if (k == "sri") {
      Rxn& r = m.rx.back(); r.sri = true;
      for (int j = 0; j < 5; ++j) r.sri_p[j] = D(t[1 + j]);
    } else if (k == "plog") {
      Rxn& r = m.rx.back();
      int n = I(t[1]);
      for (int j = 0; j < n; ++j) {
        r.plog_p.push_back(D(t[2 + 4 * j])); r.plog_A.push_back(D(t[3 + 4 * j]));
        r.plog_b.push_back(D(t[4 + 4 * j])); r.plog_E.push_back(D(t[5 + 4 * j]));
      }
    }
  }
  m.nr = (int)m.rx.size();
  return m.ns > 0;
}

// ---------------------------------------------------------------- thermo (A.1)
// Standard-state cp/R, H/(RT), S/R of species k at temperature T (Eqs. H_RT, S_R).
template <class R>
void species_thermo(const Mech& m, int k, R T, R& cp_R, R& h_RT, R& s_R) {
  const double* a = (val(T) < m.Tmid[k]) ? &m.a_lo[7 * k] : &m.a_hi[7 * k];
  cp_R = a[0] + a[1] * T + a[2] * pow(T, 2.0) + a[3] * pow(T, 3.0) + a[4] * pow(T, 4.0);
  h_RT = a[0] + a[1] / 2.0 * T + a[2] / 3.0 * pow(T, 2.0) + a[3] / 4.0 * pow(T, 3.0) + a[4] / 5.0 * pow(T, 4.0) + a[5] / T;
  s_R = a[0] * log(T) + a[1] * T + a[2] / 2.0 * pow(T, 2.0) + a[3] / 3.0 * pow(T, 3.0) + a[4] / 4.0 * pow(T, 4.0) + a[6];
}

// Gibbs energy G/(RT) of Eq. (Ck), the closed form of H/(RT) - S/R.
double gibbs_closed(const Mech& m, int k, double T) {
  const double* a = (T < m.Tmid[k]) ? &m.a_lo[7 * k] : &m.a_hi[7 * k];
  return a[0] * (1.0 - std::log(T)) - a[1] / 2.0 * T - a[2] / 6.0 * T * T - a[3] / 12.0 * T * T * T
         - a[4] / 20.0 * T * T * T * T + a[5] / T - a[6];
}

// ---------------------------------------------------------------- kinetics (A.2)
// Modified Arrhenius law, Eq. (arrhenius).
template <class R>
R arrhenius(const Arr& a, R T) { return a.A * pow(T, a.beta) * exp(-a.E / T); }

struct Detail {   // per-reaction quantities exposed for the pins
  double kf, kr, Kc, Rf, Rr, c, X, Pr, F, q;
};
const int NDET = 10;

template <class R>
R troe_F(const Rxn& r, R T, R Pr) {
  const double alpha = r.troe_p[0], T3 = r.troe_p[1], T1 = r.troe_p[2], T2 = r.troe_p[3];
  R Fcent = (1.0 - alpha) * exp(-T / T3) + alpha * exp(-T / T1) + exp(-T2 / T);
  R logFc = log10(Fcent);
  R c = -0.4 - 0.67 * logFc;
  R n = 0.75 - 1.27 * logFc;
  const double d = 0.14;
  R lp = log10(Pr);
  R f = (lp + c) / (n - d * (lp + c));
  R logF = logFc / (1.0 + f * f);
  return pow(10.0, logF);
}

template <class R>
R sri_F(const Rxn& r, R T, R Pr) {
  const double a = r.sri_p[0], b = r.sri_p[1], c = r.sri_p[2], d = r.sri_p[3], e = r.sri_p[4];
  R lp = log10(Pr);
  R X = 1.0 / (1.0 + lp * lp);
  return d * pow(T, e) * pow(a * exp(-b / T) + exp(-T / c), X);
}

// Net production rates wdot[ns] of one state (Sec. A.2); det, if given,
// receives the per-reaction quantities.
template <class R>
void production_rates(const Mech& m, R T, R p, const R* Y, R* wdot, Detail* det) {
  const int ns = m.ns;
  std::vector<R> C(ns), g(ns);
  R sigma = 0.0;
  for (int k = 0; k < ns; ++k) sigma += Y[k] / m.W[k];
  R rho = p / (R_U * T * sigma);                     // mass density, kg/m^3
  for (int k = 0; k < ns; ++k) C[k] = rho * Y[k] / m.W[k];
  for (int k = 0; k < ns; ++k) {
    R cp, h, s;
    species_thermo(m, k, T, cp, h, s);
    g[k] = h - s;                                    // G/(RT)
  }
  for (int k = 0; k < ns; ++k) wdot[k] = 0.0;
  for (int i = 0; i < m.nr; ++i) {
    const Rxn& r = m.rx[i];
    R X = 0.0;                                       // third-body concentration [X]_i
    if (r.kind == THREE_BODY || r.kind == FALLOFF || r.kind == CHEM_ACT) {
      if (r.collider >= 0) {
        X = C[r.collider];
      } else {
        for (int k = 0; k < ns; ++k) {
          double alpha = r.default_eff;
          for (auto& e : r.eff) if (e.first == k) alpha = e.second;
          X += alpha * C[k];
        }
      }
    }
    R kf = 0.0, c = 1.0, Pr = 0.0, F = 1.0;
    if (r.kind == ELEMENTARY) {
      kf = arrhenius(r.rate, T);
    } else if (r.kind == THREE_BODY) {
      kf = arrhenius(r.rate, T);
      c = X;
    } else if (r.kind == FALLOFF || r.kind == CHEM_ACT) {
      R k0 = arrhenius(r.low, T);
      R kinf = arrhenius(r.rate, T);
      Pr = k0 * X / kinf;
      if (val(Pr) < 1e-300) Pr = 1e-300;
      if (r.troe) F = troe_F(r, T, Pr);
      else if (r.sri) F = sri_F(r, T, Pr);
      if (r.kind == FALLOFF) kf = kinf * (Pr / (1.0 + Pr)) * F;
      else kf = k0 * (1.0 / (1.0 + Pr)) * F;
    } else {                                         // PLOG, Sec. A.2.3
      const size_t n = r.plog_p.size();
      double pv = val(p);
      if (pv <= r.plog_p[0]) {
        kf = arrhenius(Arr{r.plog_A[0], r.plog_b[0], r.plog_E[0]}, T);
      } else if (pv >= r.plog_p[n - 1]) {
        kf = arrhenius(Arr{r.plog_A[n - 1], r.plog_b[n - 1], r.plog_E[n - 1]}, T);
      } else {
        size_t j = 0;
        while (!(pv >= r.plog_p[j] && pv < r.plog_p[j + 1])) ++j;
        R k1 = arrhenius(Arr{r.plog_A[j], r.plog_b[j], r.plog_E[j]}, T);
        R k2 = arrhenius(Arr{r.plog_A[j + 1], r.plog_b[j + 1], r.plog_E[j + 1]}, T);
        R lk = log(k1) + (log(k2) - log(k1)) * (log(p) - std::log(r.plog_p[j])) /
                              (std::log(r.plog_p[j + 1]) - std::log(r.plog_p[j]));
        kf = exp(lk);
      }
    }
    // Equilibrium constant, Eqs. (K_p) and K_c = K_p (p_atm/(R T))^(sum nu)
    R sum_nu_g = 0.0;
    double sum_nu = 0.0;
    for (auto& e : r.prod) { sum_nu_g += e.second * g[e.first]; sum_nu += e.second; }
    for (auto& e : r.reac) { sum_nu_g = sum_nu_g - e.second * g[e.first]; sum_nu -= e.second; }
    R Kp = exp(-sum_nu_g);
    R Kc = Kp * pow(P_ATM / (R_U * T), sum_nu);
    R kr = r.reversible ? kf / Kc : R(0.0);
    // Mass-action law, Eq. (r_i)
    R Rf = kf, Rr = kr;
    for (auto& e : r.reac) Rf = Rf * pow(C[e.first], (double)e.second);
    for (auto& e : r.prod) Rr = Rr * pow(C[e.first], (double)e.second);
    R q = c * (Rf - Rr);
    for (auto& e : r.reac) wdot[e.first] = wdot[e.first] - e.second * q;
    for (auto& e : r.prod) wdot[e.first] += e.second * q;
    if (det) {
      det[i] = {val(kf), val(kr), val(Kc), val(Rf), val(Rr), val(c), val(X), val(Pr), val(F), val(q)};
    }
  }
}

// Per-point gross-rate scale max_k W_k sum_i |nu_ki| |c_i| (|Rf_i| + |Rr_i|),
// the size of the terms whose cancellation forms W_k wdot_k.
double gross_scale(const Mech& m, double T, double p, const double* Y) {
  std::vector<Detail> det(m.nr);
  std::vector<double> w(m.ns), gsum(m.ns, 0.0);
  production_rates(m, T, p, Y, w.data(), det.data());
  for (int i = 0; i < m.nr; ++i) {
    double t = std::fabs(det[i].c) * (std::fabs(det[i].Rf) + std::fabs(det[i].Rr));
    for (auto& e : m.rx[i].reac) gsum[e.first] += e.second * t;
    for (auto& e : m.rx[i].prod) gsum[e.first] += e.second * t;
  }
  double s = 0.0;
  for (int k = 0; k < m.ns; ++k) s = std::max(s, m.W[k] * gsum[k]);
  return s;
}

// ---------------------------------------------------------------- thermo mixture
void mixture_thermo(const Mech& m, double T, const double* Y, double& cp, double& h) {
  cp = 0.0; h = 0.0;
  for (int k = 0; k < m.ns; ++k) {
    double cpR, hRT, sR;
    species_thermo(m, k, T, cpR, hRT, sR);
    cp += Y[k] * cpR * R_U / m.W[k];              // c_p = sum Y_k C_p,k / W_k
    h += Y[k] * hRT * R_U * T / m.W[k];           // h = sum Y_k H_k / W_k
  }
}

// ---------------------------------------------------------------- transport (A.3)
double fit(const double* c, double L) {
  double s = 0.0;
  for (int n = 0; n < 5; ++n) s += c[n] * std::pow(L, (double)n);
  return s;
}

// The same polynomial summed in long double: direct fits of eta, lambda and
// 1/D_kj have condition numbers up to ~1e6 in the monomial basis of ln T, so
// a float64 sum would carry ~1e-10 of rounding; extended precision keeps the
// oracle's own error below the 1e-12 bar.
double fit_ext(const double* c, double L) {
  long double s = 0.0L;
  for (int n = 0; n < 5; ++n) s += (long double)c[n] * std::pow((long double)L, (long double)n);
  return (double)s;
}

// Pure-species properties from the fits in ln T (Sec. A.3.4): of ln eta,
// ln lambda and ln D_kj, exponentiated; or, with direct fits, of eta and
// lambda themselves and of the reciprocal 1/D_kj (the paper evaluates the
// reciprocal polynomial of the binary diffusion coefficients, Sec. 2.3.2).
void species_transport(const Mech& m, double T, double p, double* eta, double* lam, double* Dkj) {
  const double L = std::log(T);
  for (int k = 0; k < m.ns; ++k) {
    eta[k] = m.direct ? fit_ext(&m.eta[5 * k], L) : std::exp(fit(&m.eta[5 * k], L));
    lam[k] = m.direct ? fit_ext(&m.lam[5 * k], L) : std::exp(fit(&m.lam[5 * k], L));
  }
  if (Dkj)
    for (int k = 0; k < m.ns; ++k)
      for (int j = 0; j < m.ns; ++j) {
        const double* c = &m.dif[5 * (k * m.ns + j)];
        Dkj[k * m.ns + j] = (m.direct ? 1.0 / fit_ext(c, L) : std::exp(fit(c, L))) * P_ATM / p;
      }
}

// Wilke/Bird interaction factor phi_kj.  The molecular-weight ratio inside
// the quarter power is W_j/W_k, the standard form, for which
// phi_jk = phi_kj (eta_j/eta_k)(W_k/W_j); the appendix display prints the
// ratio inverted, which breaks that reciprocity.
double wilke_phi(const Mech& m, const double* eta, int k, int j) {
  return 1.0 / std::sqrt(8.0) * std::pow(1.0 + m.W[k] / m.W[j], -0.5) *
         std::pow(1.0 + std::pow(eta[k] / eta[j], 0.5) * std::pow(m.W[j] / m.W[k], 0.25), 2.0);
}

void mixture_transport(const Mech& m, double T, double p, const double* Y, double& mu, double& lambda, double* Dk) {
  const int ns = m.ns;
  std::vector<double> eta(ns), lam(ns), Dkj(ns * ns), X(ns);
  species_transport(m, T, p, eta.data(), lam.data(), Dkj.data());
  double sigma = 0.0;
  for (int k = 0; k < ns; ++k) sigma += Y[k] / m.W[k];
  for (int k = 0; k < ns; ++k) X[k] = (Y[k] / m.W[k]) / sigma;
  double Wbar = 0.0;
  for (int k = 0; k < ns; ++k) Wbar += X[k] * m.W[k];
  // Wilke viscosity with the Bird et al. phi_kj
  mu = 0.0;
  for (int k = 0; k < ns; ++k) {
    double den = 0.0;
    for (int j = 0; j < ns; ++j) den += X[j] * wilke_phi(m, eta.data(), k, j);
    mu += X[k] * eta[k] / den;
  }
  // Mathur conductivity
  double s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < ns; ++k) { s1 += X[k] * lam[k]; s2 += X[k] / lam[k]; }
  lambda = 0.5 * (s1 + 1.0 / s2);
  // mixture-averaged diffusion, Eq. (mix_diff)
  for (int k = 0; k < ns; ++k) {
    double s = 0.0;
    for (int j = 0; j < ns; ++j)
      if (j != k) s += X[j] / Dkj[k * ns + j];
    Dk[k] = (s > 0.0) ? (Wbar - X[k] * m.W[k]) / Wbar / s : Dkj[k * ns + k];
  }
}

template <class F>
void parallel(long n, int nthreads, F fn) {
  if (nthreads <= 1 || n < 2) { fn(0L, n); return; }
  std::vector<std::thread> th;
  long chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    long a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back(fn, a, b);
  }
  for (auto& x : th) x.join();
}

}  // namespace

// ---------------------------------------------------------------- C entry points
extern "C" {

int ora_load(const char* path, void** out) {
  Mech* m = new Mech();
  std::string err;
  if (!parse(path, *m, err)) { delete m; std::fprintf(stderr, "oracle: %s: %s\n", path, err.c_str()); return 1; }
  *out = m;
  return 0;
}

void ora_free(void* h) { delete static_cast<Mech*>(h); }

int ora_sizes(void* h, int* ns, int* nr) {
  Mech* m = static_cast<Mech*>(h);
  *ns = m->ns; *nr = m->nr;
  return 0;
}

int ora_ndetail() { return NDET; }

int ora_species_thermo(void* h, double T, double* cp_R, double* h_RT, double* s_R, double* g_RT, double* g_closed) {
  Mech& m = *static_cast<Mech*>(h);
  for (int k = 0; k < m.ns; ++k) {
    species_thermo(m, k, T, cp_R[k], h_RT[k], s_R[k]);
    g_RT[k] = h_RT[k] - s_R[k];
    g_closed[k] = gibbs_closed(m, k, T);
  }
  return 0;
}

// Y is species-major [ns][ld]; wdot likewise.
int ora_production_rates(void* h, const double* T, const double* p, const double* Y, long ld,
                         double* wdot, long n, int nthreads) {
  Mech& m = *static_cast<Mech*>(h);
  parallel(n, nthreads, [&](long a, long b) {
    std::vector<double> y(m.ns), w(m.ns);
    for (long i = a; i < b; ++i) {
      for (int k = 0; k < m.ns; ++k) y[k] = Y[k * ld + i];
      production_rates(m, T[i], p[i], y.data(), w.data(), (Detail*)nullptr);
      for (int k = 0; k < m.ns; ++k) wdot[k * ld + i] = w[k];
    }
  });
  return 0;
}

// Rates of progress q_i = c_i (k_f prod C^nu' - k_r prod C^nu'') of every
// reaction, [nr][ld] reaction-major.
int ora_rates_of_progress(void* h, const double* T, const double* p, const double* Y, long ld, double* q,
                          long n, int nthreads) {
  Mech& m = *static_cast<Mech*>(h);
  parallel(n, nthreads, [&](long a, long b) {
    std::vector<double> y(m.ns), w(m.ns);
    std::vector<Detail> det(m.nr);
    for (long i = a; i < b; ++i) {
      for (int k = 0; k < m.ns; ++k) y[k] = Y[k * ld + i];
      production_rates(m, T[i], p[i], y.data(), w.data(), det.data());
      for (int r = 0; r < m.nr; ++r) q[r * ld + i] = det[r].q;
    }
  });
  return 0;
}

// Per-reaction gross scale |c_i| max(|k_f prod C^nu'|, |k_r prod C^nu''|),
// [nr][ld]: the size of the two terms whose difference is q_i.
int ora_reaction_gross(void* h, const double* T, const double* p, const double* Y, long ld, double* out,
                       long n, int nthreads) {
  Mech& m = *static_cast<Mech*>(h);
  parallel(n, nthreads, [&](long a, long b) {
    std::vector<double> y(m.ns), w(m.ns);
    std::vector<Detail> det(m.nr);
    for (long i = a; i < b; ++i) {
      for (int k = 0; k < m.ns; ++k) y[k] = Y[k * ld + i];
      production_rates(m, T[i], p[i], y.data(), w.data(), det.data());
      for (int r = 0; r < m.nr; ++r) out[r * ld + i] = std::fabs(det[r].c) * std::max(std::fabs(det[r].Rf), std::fabs(det[r].Rr));
    }
  });
  return 0;
}

int ora_reaction_detail(void* h, double T, double p, const double* Y, double* out) {
  Mech& m = *static_cast<Mech*>(h);
  std::vector<double> w(m.ns);
  std::vector<Detail> det(m.nr);
  production_rates(m, T, p, Y, w.data(), det.data());
  std::memcpy(out, det.data(), sizeof(Detail) * m.nr);
  return 0;
}

int ora_gross_scale(void* h, const double* T, const double* p, const double* Y, long ld, double* scale,
                    long n, int nthreads) {
  Mech& m = *static_cast<Mech*>(h);
  parallel(n, nthreads, [&](long a, long b) {
    std::vector<double> y(m.ns);
    for (long i = a; i < b; ++i) {
      for (int k = 0; k < m.ns; ++k) y[k] = Y[k * ld + i];
      scale[i] = gross_scale(m, T[i], p[i], y.data());
    }
  });
  return 0;
}

int ora_thermo(void* h, const double* T, const double* p, const double* Y, long ld, double* cp, double* hm,
               long n, int nthreads) {
  Mech& m = *static_cast<Mech*>(h);
  (void)p;
  parallel(n, nthreads, [&](long a, long b) {
    std::vector<double> y(m.ns);
    for (long i = a; i < b; ++i) {
      for (int k = 0; k < m.ns; ++k) y[k] = Y[k * ld + i];
      mixture_thermo(m, T[i], y.data(), cp[i], hm[i]);
    }
  });
  return 0;
}

int ora_species_transport(void* h, double T, double p, double* eta, double* lam, double* Dkj) {
  Mech& m = *static_cast<Mech*>(h);
  species_transport(m, T, p, eta, lam, Dkj);
  return 0;
}

int ora_wilke_phi(void* h, double T, double* phi) {
  Mech& m = *static_cast<Mech*>(h);
  std::vector<double> eta(m.ns), lam(m.ns);
  species_transport(m, T, P_ATM, eta.data(), lam.data(), nullptr);
  for (int k = 0; k < m.ns; ++k)
    for (int j = 0; j < m.ns; ++j) phi[k * m.ns + j] = wilke_phi(m, eta.data(), k, j);
  return 0;
}

int ora_transport(void* h, const double* T, const double* p, const double* Y, long ld, double* mu, double* lam,
                  double* Dk, long n, int nthreads) {
  Mech& m = *static_cast<Mech*>(h);
  parallel(n, nthreads, [&](long a, long b) {
    std::vector<double> y(m.ns), d(m.ns);
    for (long i = a; i < b; ++i) {
      for (int k = 0; k < m.ns; ++k) y[k] = Y[k * ld + i];
      mixture_transport(m, T[i], p[i], y.data(), mu[i], lam[i], d.data());
      for (int k = 0; k < m.ns; ++k) Dk[k * ld + i] = d[k];
    }
  });
  return 0;
}

// Dense Jacobian of one state at fixed p: J[k][0] = d wdot_k / dT,
// J[k][1 + j] = d wdot_k / dY_j, by forward-mode dual numbers (one seed
// direction per column).
int ora_jacobian(void* h, double T, double p, const double* Y, double* J) {
  Mech& m = *static_cast<Mech*>(h);
  const int ns = m.ns;
  std::vector<Dual> y(ns), w(ns);
  for (int col = 0; col <= ns; ++col) {
    Dual t(T, col == 0 ? 1.0 : 0.0);
    for (int k = 0; k < ns; ++k) y[k] = Dual(Y[k], col == k + 1 ? 1.0 : 0.0);
    production_rates(m, t, Dual(p, 0.0), y.data(), w.data(), (Detail*)nullptr);
    for (int k = 0; k < ns; ++k) J[k * (ns + 1) + col] = w[k].d;
  }
  return 0;
}

}  // extern "C"
