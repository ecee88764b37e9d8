"""GB300-native SPH hot path (placeholder; the binding is added with the C-ABI)."""
