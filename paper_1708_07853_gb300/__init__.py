"""GB300 (sm_103a) 2-D discrete wavelet transform by non-separable lifting."""
