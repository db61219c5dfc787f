// rect_f32mm.cu — rectangular executor instantiated for FP32 max / min.
#include "rect_launch.cuh"

namespace hp {
hp_status launch_rect_f32_max(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpF32Max>(np, cfg, a);
}
hp_status launch_rect_f32_min(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpF32Min>(np, cfg, a);
}
}  // namespace hp
