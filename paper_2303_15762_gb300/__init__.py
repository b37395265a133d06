"""GB300-native backward path tracing of generalized rays (arXiv 2303.15762)."""
