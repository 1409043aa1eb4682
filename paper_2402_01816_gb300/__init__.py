"""GB300-native stable mergesort after the greeNsort method (placeholder; the
binding is added with the CUDA library)."""
