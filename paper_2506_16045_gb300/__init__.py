"""GB300-native SGN constraint-solve library (Python binding over the C ABI)."""
