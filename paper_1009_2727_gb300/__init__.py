"""GB300-native boosted-frame PIC step (placeholder; the binding is added with the CUDA library)."""
