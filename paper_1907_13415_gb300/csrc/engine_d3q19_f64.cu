// Engine instantiation: LatD3Q19 lattice, double arithmetic.
#include "engine.cuh"

namespace nlc {
std::unique_ptr<EngineBase> make_engine_d3q19_f64(const EngineArgs& a, nlc_status* st,
                                          std::string* msg) {
  return make_engine<LatD3Q19, double>(a, st, msg);
}
}  // namespace nlc
