// Autotuner cache: for each (GPU, kernel family, angular momentum, size
// bucket) the launch variant that ran fastest in a timed trial.  Process-wide
// and thread-safe; a trial runs once per key, on the first call that needs it.
#pragma once

namespace pcm {

enum TuneKind {
    TUNE_ESP_PPT = 0,    // FP32 ESP kernel: pair-driven with 4 (0) or 2 (1) points per thread, or MS-driven (2)
    TUNE_FOCK_NPT = 1,   // FP32 Fock kernel: primitive pairs per thread (1 or 2)
    // the same choices for the kernels with scalar FP32 instructions (pcm_options.fp32x2 = 0)
    TUNE_ESP_PPT_SCALAR = 2,
    TUNE_FOCK_NPT_SCALAR = 3,
    // the packed ESP blocks of a batch, which run in one launch for all molecules: pair-driven
    // with 4 (0) or 2 (1) points per thread (the per-molecule MS-driven kernel has no batched form)
    TUNE_ESP_PPT_BATCH = 4,
};

// size bucket of a kernel's work: floor(log2(n)) (pairs of the class)
int tune_bucket(long long n);
// the remembered choice, or -1
int tune_get(int device, int kind, int L, int bucket);
// remember a choice with the trial times of up to three variants (ms; 0: not tried)
void tune_set(int device, int kind, int L, int bucket, int choice, float ms0, float ms1, float ms2 = 0.f);
// copy up to max records of (device, kind, L, bucket, choice, trial microseconds of variants 0, 1, 2)
// into out (8 ints each); returns the count
int tune_table(int *out, int max);

}  // namespace pcm
