// FP64 instantiation of the FETI-DP engine.
#include "engine_impl.cuh"

namespace schur {
EngineBase* make_engine_f64(const HostMaps* hm, const DevMaps* dm, double gamma, double sre) {
  return new Engine<double>(hm, dm, gamma, sre);
}
}  // namespace schur
