// keys_min_dna64.cu -- the DNA form of the single-pass minimizer kernel (keys_min.cuh) with 64-bit keys
// (16 < k <= 29) without barriers, instantiated for window lengths 4..17 in a translation unit of its own.
#include "keys_min.cuh"

namespace sws {
namespace keysmin {

cudaError_t launch_dna64_none(const KeysArgs &a, int w, int num_sms, cudaStream_t st) {
  CUtensorMap none{};  // the DNA form has no tensor map
  switch (w) {
    case 4: return launch_w_keys<4, true, KB_NONE, true>(none, a, num_sms, st);
    case 5: return launch_w_keys<5, true, KB_NONE, true>(none, a, num_sms, st);
    case 6: return launch_w_keys<6, true, KB_NONE, true>(none, a, num_sms, st);
    case 7: return launch_w_keys<7, true, KB_NONE, true>(none, a, num_sms, st);
    case 8: return launch_w_keys<8, true, KB_NONE, true>(none, a, num_sms, st);
    case 9: return launch_w_keys<9, true, KB_NONE, true>(none, a, num_sms, st);
    case 10: return launch_w_keys<10, true, KB_NONE, true>(none, a, num_sms, st);
    case 11: return launch_w_keys<11, true, KB_NONE, true>(none, a, num_sms, st);
    case 12: return launch_w_keys<12, true, KB_NONE, true>(none, a, num_sms, st);
    case 13: return launch_w_keys<13, true, KB_NONE, true>(none, a, num_sms, st);
    case 14: return launch_w_keys<14, true, KB_NONE, true>(none, a, num_sms, st);
    case 15: return launch_w_keys<15, true, KB_NONE, true>(none, a, num_sms, st);
    case 16: return launch_w_keys<16, true, KB_NONE, true>(none, a, num_sms, st);
    case 17: return launch_w_keys<17, true, KB_NONE, true>(none, a, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace keysmin
}  // namespace sws
