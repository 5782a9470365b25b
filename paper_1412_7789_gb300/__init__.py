"""GB300-native failureless Aho-Corasick (PFAC) matching."""
