// Internal declarations of the kx library: the mechanism model read from a
// KXMECH file, the CUDA source emitter and its per-point operation counts.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/kx.h"

namespace kx {

constexpr double R_U = 8314.46261815324;   // J/(kmol K)
constexpr double P_ATM = 101325.0;         // Pa

struct Arrh {
  double A = 0.0, beta = 0.0, E = 0.0;      // k = A T^beta exp(-E/T), E in K
};

enum class Kind { Elementary, ThreeBody, Falloff, ChemAct, Plog };
enum class Blend { Lindemann, Troe, Sri };

struct Reaction {
  Kind kind = Kind::Elementary;
  bool reversible = true;
  std::vector<std::pair<int, int>> reac, prod;   // (species, stoichiometric coefficient)
  Arrh k;                                        // k_f, k_inf (falloff) or k_inf (chem. activated)
  Arrh k0;                                       // k_0 of falloff / chemically activated reactions
  bool has_k0 = false;
  double default_eff = 1.0;
  std::vector<std::pair<int, double>> eff;       // third-body efficiencies that differ from default
  int collider = -1;                             // single-species third body, or -1
  Blend blend = Blend::Lindemann;
  double troe[4] = {0, 0, 0, 0};                 // alpha, T***, T*, T**
  double sri[5] = {0, 0, 0, 1, 0};               // a, b, c, d, e
  std::vector<std::array<double, 4>> plog;       // (p [Pa], A, beta, E), ascending p
  bool third_body() const { return kind == Kind::ThreeBody || kind == Kind::Falloff || kind == Kind::ChemAct; }
};

struct Mechanism {
  std::string name;
  std::vector<std::string> elements;
  int ns = 0;
  std::vector<std::string> species;
  std::vector<double> W;                 // kg/kmol
  std::vector<int> comp;                 // [ns][n_elements]
  std::vector<char> inert;
  std::vector<double> Tlow, Tmid, Thigh;
  std::vector<double> a_lo, a_hi;        // [ns][7] NASA-7
  std::vector<double> eta, lam;          // [ns][5]: ln eta, ln lambda as polynomials in ln T
  std::vector<double> dif;               // [ns][ns][5]: ln D_jk at p_atm
  bool fit_direct = false;               // eta, lam, dif hold fits of eta, lambda and 1/D_jk themselves
  std::vector<Reaction> rx;
  int nr() const { return (int)rx.size(); }
};

// Parse and validate a KXMECH 1 file.  Returns KX_OK or an error code with a message.
kx_status parse_mechanism(const std::string& path, Mechanism& m, std::string& err);

enum class KernelKind { Wdot, Rop, Thermo, Transport, Vjp };

struct EmitOptions {
  bool mixed = false;       // float32 bulk arithmetic
  int diff_mode = 1;        // 1 symmetric pairs, 2 full matrix
  int kc_mode = 0;          // 0 log space, 1 per-species exponential products
  int tr_mode = 0;          // float64 transport: 0 double-float on the float32 pipe, 1 native float64
  int tr_layout = 3;        // transport species vectors: 1 all in shared memory, 2 X in local memory, 3 all local
  int block = 128;
  int part = 0;             // transport: 0 all outputs, 1 viscosity and conductivity, 2 diffusion
  int maxrreg = 0;          // register cap per thread (0: compiler choice)
  int rates_mode = 0;       // 0 auto, 1 unrolled, 2 table driven (large mechanisms)
  int rates_arith = 0;      // float64-accurate rates: 0/2 double-float (reaction classes), 1 native float64
  bool scratch = false;     // float-pair rates: species vectors in a global scratch array passed by the
                            // caller (strided by the grid's thread count) instead of local memory
  int rates_layout = 0;     // float-pair production rates: 0/1 thread per state, 2 warp-cooperative (the
                            // states of a warp share its lanes, species vectors in shared memory)
  int rates_group = 0;      // warp-cooperative: states per warp (power of two up to 32; 0: one)
  int vjp_form = 0;         // double-float adjoint, d/dC_k: 0 rate mantissa times a per-state reciprocal
                            // concentration, 1 one log-space exponential per entry
  int vjp_layout = 0;       // double-float adjoint: 0/1 thread per state, 2 warp-cooperative
  int rates_negligible = 0; // double-float rates: 0 float32 for reactions negligible in every state of a warp, 1 never
};

// Launch shape of the warp-cooperative production-rate kernel.
struct WcShape {
  int states_per_warp = 1, states_per_block = 1, smem_per_block = 0;
  double lane_use = 1.0;   // (state, reaction) pairs over lane slots of the class rounds
};
bool wdot_is_wc(const Mechanism& m, KernelKind kind, const EmitOptions& opt);
bool vjp_is_wc(const Mechanism& m, KernelKind kind, const EmitOptions& opt);
int vjp_wc_smem(const Mechanism& m, const EmitOptions& opt);   // dynamic shared memory per block
WcShape wdot_wc_shape(const Mechanism& m, const EmitOptions& opt);

// Operation counts per point, tallied while emitting (library calls such as
// exp and log counted once each, in their own columns).
struct OpCounts {
  double fp64 = 0, fp32 = 0, exp64 = 0, log64 = 0, div64 = 0, exp32 = 0, log32 = 0, div32 = 0;
};

// CUDA C++ source of one kernel, entry point named `entry`.
std::string emit_kernel(const Mechanism& m, KernelKind kind, const EmitOptions& opt, const std::string& entry,
                        OpCounts* counts);

// Global scratch bytes per thread of the float-pair rate kernel built with
// EmitOptions::scratch ({ln |C|, mu} float4 and a float-pair accumulator per species).
inline int rates_scratch_per_thread(const Mechanism& m) { return 24 * m.ns; }

// Dynamic shared memory per thread that a kernel of this kind needs.
int transport_smem_per_thread(const Mechanism& m, bool mixed, int part, int layout);

// Device-side helper functions prepended to every generated kernel.
extern const char* kDevicePrelude;

}  // namespace kx
