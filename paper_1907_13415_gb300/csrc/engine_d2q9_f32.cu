// Engine instantiation: LatD2Q9 lattice, float arithmetic.
#include "engine.cuh"

namespace nlc {
std::unique_ptr<EngineBase> make_engine_d2q9_f32(const EngineArgs& a, nlc_status* st,
                                          std::string* msg) {
  return make_engine<LatD2Q9, float>(a, st, msg);
}
}  // namespace nlc
