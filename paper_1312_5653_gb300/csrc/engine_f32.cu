// Complex FP32 instantiation of the FETI-DP engine (the inner solver of the mixed-precision form).
#include "engine_impl.cuh"

namespace schur {
EngineBase* make_engine_f32(const HostMaps* hm, const DevMaps* dm, double gamma, double sre) {
  return new Engine<float>(hm, dm, gamma, sre);
}
}  // namespace schur
