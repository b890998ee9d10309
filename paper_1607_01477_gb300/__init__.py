"""GB300-native blocked multi-shift triangular solves (arXiv:1607.01477)."""
