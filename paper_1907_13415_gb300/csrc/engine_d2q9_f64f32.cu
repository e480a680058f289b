// Engine instantiation: LatD2Q9 lattice, double arithmetic and Q, float
// populations (the FP32-population, FP64-Q precision).
#include "engine.cuh"

namespace nlc {
std::unique_ptr<EngineBase> make_engine_d2q9_f64f32(const EngineArgs& a, nlc_status* st,
                                                std::string* msg) {
  return make_engine<LatD2Q9, double, float>(a, st, msg);
}
}  // namespace nlc
