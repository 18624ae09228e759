"""GB300-native bulk histogram filling (ROOT axis semantics) behind a C ABI."""
