"""GB300-native Monte Carlo path tracer (CUDA, sm_103a) behind a small C-ABI."""
