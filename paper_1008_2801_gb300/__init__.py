"""GB300-native variable-coefficient multigrid Poisson solver (placeholder)."""
