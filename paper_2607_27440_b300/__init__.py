"""B300-native kLST shift-and-invert eigensolve (Python binding over the C-ABI library)."""
