// Filter bank, adjoints and morphology subgradient entry points.
#include "hp_internal.h"

using namespace hp;

extern "C" {

int hp_filterbank3d(const hp_volume*, hp_volume* const*, const hp_filter*, int, void*) {
  return set_error(HP_ERR_UNSUPPORTED, "filter bank not built yet");
}
int hp_filterbank3d_bricks(const hp_volume*, hp_volume* const*, const hp_filter*, int,
                           const hp_box*, int, void*) {
  return set_error(HP_ERR_UNSUPPORTED, "filter bank not built yet");
}
int hp_filterbank3d_adjoint(const hp_volume*, const hp_volume* const*, const hp_filter*, int,
                            hp_volume*, void*) {
  return set_error(HP_ERR_UNSUPPORTED, "adjoint not built yet");
}
int hp_morph3d_backward(const hp_volume*, const hp_volume*, int, hp_se, int, hp_volume*, void*) {
  return set_error(HP_ERR_UNSUPPORTED, "morphology backward not built yet");
}
int hp_release_cache(void) { return HP_OK; }

}  // extern "C"
