// Engine instantiation: LatD2Q9 lattice, double arithmetic.
#include "engine.cuh"

namespace nlc {
std::unique_ptr<EngineBase> make_engine_d2q9_f64(const EngineArgs& a, nlc_status* st,
                                          std::string* msg) {
  return make_engine<LatD2Q9, double>(a, st, msg);
}
}  // namespace nlc
