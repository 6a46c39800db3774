"""CPU FP64 oracle (test infrastructure only; see ipa_oracle)."""
