// Engine instantiation: LatD3Q19 lattice, float arithmetic.
#include "engine.cuh"

namespace nlc {
std::unique_ptr<EngineBase> make_engine_d3q19_f32(const EngineArgs& a, nlc_status* st,
                                          std::string* msg) {
  return make_engine<LatD3Q19, float>(a, st, msg);
}
}  // namespace nlc
