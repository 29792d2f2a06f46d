// Learned initial guess.
#include "mpfc_internal.h"

bool mpfc_has_guess_model(const mpfc_s* H) { return H && H->guess_model; }
void mpfc_enqueue_learned_guess(mpfc_s* H, cudaStream_t s) { (void)H; (void)s; }
