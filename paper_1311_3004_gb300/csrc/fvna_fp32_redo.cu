// fvna_fp32_redo.cu -- the second kernel of each binary32 sweep: the tiles
// whose speculative march met a face that is not subsonic, marched again
// with the general fluctuation split (same source as fvna_fp32.cu, built
// as its own unit so the two compile in parallel).
#define FVNA_REDO true
#define FVNA_REDO_UNIT 1
#define FVNA_CHECK_SYMBOL fvna_check_word_redo
#include "fvna_fp32.cu"
