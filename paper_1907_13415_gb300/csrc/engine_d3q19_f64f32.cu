// Engine instantiation: LatD3Q19 lattice, double arithmetic and Q, float
// populations (the FP32-population, FP64-Q precision).
#include "engine.cuh"

namespace nlc {
std::unique_ptr<EngineBase> make_engine_d3q19_f64f32(const EngineArgs& a, nlc_status* st,
                                                std::string* msg) {
  return make_engine<LatD3Q19, double, float>(a, st, msg);
}
}  // namespace nlc
