"""GB300-native two-component pseudopotential LBM (arXiv 2505.22256)."""
