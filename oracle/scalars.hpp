// Test infrastructure: scalar types that the FP64 CPU oracle is instantiated with.
//
// The oracle's step is written once, generically over its scalar type T.  This file
// provides the non-double instantiations:
//   Dual    forward-mode derivative (value, one tangent) -> J v  without any hand derivation;
//   TVar    reverse-mode derivative through a recorded tape -> J^T w, likewise generic;
//   Counted a double that counts arithmetic operations, to measure flops per cell.
// Comparisons (limiter branches, HLLC wave-speed branches, floors) are taken on values, so a
// derivative is the derivative of the branch the value selected.
//
// Only the tests, the smoke check and the timed CPU baseline use anything under oracle/.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace oracle {

inline double value(double x) { return x; }
inline double sqrt(double x) { return std::sqrt(x); }

// ---------------------------------------------------------------- Dual (forward mode)
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline double value(const Dual& a) { return a.v; }
inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt(const Dual& a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}

// ---------------------------------------------------------------- TVar (reverse mode)
// A node records up to two parents and the partial derivative with respect to each.
struct TapeNode {
  int32_t a, b;
  double da, db;
};
struct Tape {
  std::vector<TapeNode> nodes;
  int32_t push(int32_t a, double da, int32_t b, double db) {
    nodes.push_back(TapeNode{a, b, da, db});
    return (int32_t)nodes.size() - 1;
  }
  // Leaf (independent variable): a node with no parents.
  int32_t leaf() { return push(-1, 0.0, -1, 0.0); }
  // Reverse sweep: adj must have nodes.size() entries, seeded at the outputs.
  void reverse(std::vector<double>& adj) const {
    for (int64_t i = (int64_t)nodes.size() - 1; i >= 0; --i) {
      const TapeNode& n = nodes[(size_t)i];
      double g = adj[(size_t)i];
      if (g == 0.0) continue;
      if (n.a >= 0) adj[(size_t)n.a] += n.da * g;
      if (n.b >= 0) adj[(size_t)n.b] += n.db * g;
    }
  }
};
// The tape that TVar operations record onto (one oracle call at a time, single thread).
inline Tape*& active_tape() {
  static thread_local Tape* t = nullptr;
  return t;
}

struct TVar {
  double v;
  int32_t i;  // tape index, -1 for a constant
  TVar() : v(0), i(-1) {}
  TVar(double x) : v(x), i(-1) {}
  TVar(double x, int32_t idx) : v(x), i(idx) {}
};
inline double value(const TVar& a) { return a.v; }
inline TVar tv_make(double v, int32_t a, double da, int32_t b, double db) {
  if (a < 0 && b < 0) return TVar(v);
  return TVar(v, active_tape()->push(a, da, b, db));
}
inline TVar operator+(const TVar& a, const TVar& b) { return tv_make(a.v + b.v, a.i, 1.0, b.i, 1.0); }
inline TVar operator-(const TVar& a, const TVar& b) { return tv_make(a.v - b.v, a.i, 1.0, b.i, -1.0); }
inline TVar operator-(const TVar& a) { return tv_make(-a.v, a.i, -1.0, -1, 0.0); }
inline TVar operator*(const TVar& a, const TVar& b) { return tv_make(a.v * b.v, a.i, b.v, b.i, a.v); }
inline TVar operator/(const TVar& a, const TVar& b) {
  double q = a.v / b.v;
  return tv_make(q, a.i, 1.0 / b.v, b.i, -q / b.v);
}
inline TVar sqrt(const TVar& a) {
  double s = std::sqrt(a.v);
  return tv_make(s, a.i, 0.5 / s, -1, 0.0);
}

// ---------------------------------------------------------------- Counted (op counting)
// Counts binary +, -, *, / and sqrt (each 1).  Sign flips, comparisons and selections are
// not arithmetic and are not counted.
inline uint64_t& op_counter() {
  static thread_local uint64_t c = 0;
  return c;
}
// The same operations by kind: [0] + and -, [1] *, [2] /, [3] sqrt.
inline uint64_t* op_kinds() {
  static thread_local uint64_t k[4] = {0, 0, 0, 0};
  return k;
}
struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double x) : v(x) {}
};
inline double value(const Counted& a) { return a.v; }
inline Counted operator+(const Counted& a, const Counted& b) { ++op_counter(); ++op_kinds()[0]; return Counted(a.v + b.v); }
inline Counted operator-(const Counted& a, const Counted& b) { ++op_counter(); ++op_kinds()[0]; return Counted(a.v - b.v); }
inline Counted operator-(const Counted& a) { return Counted(-a.v); }  // sign flip: free
inline Counted operator*(const Counted& a, const Counted& b) { ++op_counter(); ++op_kinds()[1]; return Counted(a.v * b.v); }
inline Counted operator/(const Counted& a, const Counted& b) { ++op_counter(); ++op_kinds()[2]; return Counted(a.v / b.v); }
inline Counted sqrt(const Counted& a) { ++op_counter(); ++op_kinds()[3]; return Counted(std::sqrt(a.v)); }

}  // namespace oracle
